// sbi_host.cu - C ABI, context, pass planner and step graph of the ESBI hot path.
//
// One right-hand-side (RHS) evaluation for a group of equal-grid members is
// planned once as a fixed chain of passes (see sbi_internal.h for layouts):
//
//   Col A      F{phi~}, F{eta}  ->  V_1 = k tanh(kh) phi^, grad phi~, grad eta,
//              grad varphi_1 = ik sech(kh) phi^                (Sec. 2.4, order 1)
//   Row l      inverse x-FFT of V_{l-1} (and grad phi~ at l = 2, grad varphi_{l-1}),
//              then every product that later orders need from it:
//              eta^j V_{l-1}, eta^j grad phi~, delta^j grad varphi_{l-1}
//   Col l      sum of the order-l terms of F{V_l} and F{varphi_l}
//              (Appendix C; coefficient table in plan_col_level), masked
//   Row RHS    V = sum_l V_l, grad eta, grad phi~ -> dynamic condition
//              (Eq. prognostic) and the damping products w grad phi~ (Eq. pd)
//   Col RHS    dealias the dynamic condition, add the damping pressure
//   RK s       classical RK4 stage in FP64; next stage's working copies
//
// Each product is formed from the freshly inverted order as soon as that order
// exists ("eager" products), so no physical V_l is stored or re-read.  A step is
// four RHS evaluations plus the RK passes, and, with the low-pass filter on, a
// projection of the FP64 state.  The whole step is captured into a CUDA graph
// per dt and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <list>
#include <map>
#include <string>
#include <vector>

#include "../../include/sbi.h"
#include "fft.cuh"
#include "sbi_internal.h"
#include "schedule.h"

using namespace sbi;

namespace {

std::string g_create_error = "no error";

enum PassKind { PK_ROW = 0, PK_COL = 1, PK_RK = 2, PK_CONV = 3, PK_WMK = 4, PK_NORM = 5 };

// Cash-Karp 5(4) pair (the adaptive integrating factor): nodes, stage
// weights, order-5 and order-4 solution weights
constexpr double kCkC[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
constexpr double kCkA[6][5] = {{0, 0, 0, 0, 0},
                               {1.0 / 5.0, 0, 0, 0, 0},
                               {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
                               {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
                               {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
                               {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0,
                                253.0 / 4096.0}};
constexpr double kCkB5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
constexpr double kCkB4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                             277.0 / 14336.0, 1.0 / 4.0};

// Step norms of the adaptive scheme: per member, over the kept modes,
// |Ee|^2, |Ep|^2, |eta^|^2, |phi^|^2 (Parseval weights 1 for kx = 0, 2 else)
struct NormParams {
  const void *ee, *ep, *ue, *up;
  long long stride;   // complex elements per member
  int W, ny, n;
  double* part;       // [n][kConvBlocks][4]
  double* out;        // [n][4]
};

// Device-side convergence test of the adaptive order (opt.adapt_tol > 0):
// after order l, per member, inc = ||F{V_l}||^2 and tot = ||F{V_1 + .. + V_l}||^2
// (Parseval on the mixed layout, FP64).  A member still iterating whose
// inc <= tol^2 tot stops: its mixed sum is written to Vsum and its flag cleared,
// so the passes of the higher orders skip it.
constexpr int kConvBlocks = 64;   // partial sums per member
struct ConvParams {
  int phase;            // 0: reset flags, 1: partial norms, 2: write sums, 3: update flags
  int nlev;             // l: buffers V_1..V_l
  const void* V[7];
  void* vsum;
  long long stride;     // complex elements per member
  int W, ny, n, level, last;
  double tol2;
  int *conv, *orders, *notconv;
  double* red;          // [n][kConvBlocks][2]
};
// Pneumatic wavemaker: the surface pressure profile along x at one stage
// time, out[x] = sum_j prof[j][x] sin(omega_j t_s + theta_j), t_s = *t + offset.
struct WmkParams {
  const double* prof;    // [J][nx] FP64 bells g a_j C_j exp(-(k_j d)^2 / 2)
  const double* omega;   // [J]
  const double* phase;   // [J]
  const double* t;       // simulation time of the step start (device)
  double offset;         // stage time minus step start
  void* out;             // nx reals in the working precision
  int J, nx;
};
enum Family { FAM_COL = 0, FAM_ROW = 1, FAM_RK = 2, FAM_CONV = 3, FAM_WMK = 4, FAM_COUNT = 5 };
const char* kFamilyNames[FAM_COUNT] = {"k_col (column FFT + spectral combine)",
                                       "k_row (row FFT + products)", "k_rk (RK4 stage)",
                                       "k_conv (adaptive-order test / step norms)",
                                       "k_wavemaker (surface pressure profile)"};

struct Pass {
  PassKind kind;
  int nsize;  // nx for row / rk passes, ny for column passes
  RowParams row;
  ColParams col;
  RkParams rk;
  ConvParams conv;
  WmkParams wmk;
  NormParams norm;
  double bytes;   // algorithmic device-memory traffic of the launch
  double xforms;  // 1-D transform passes over a whole field, times the field's points
};

// A table whose values depend on the step h: tau = r h, coefficient c0 h^p.
struct DynTable {
  void* ptr;
  TableSpec spec;
  double r;
  int p;
};

struct Group {
  int nx = 0, ny = 0, W = 0, n = 0;
  double Lx = 0, Ly = 0, h0 = 0;
  bool variable = false, deep = false, two_d = false;
  int kx_keep = 0, ky_keep = 0;
  std::vector<int> members;  // context member ids
  double *eta0 = nullptr, *phi0 = nullptr, *acc_eta = nullptr, *acc_phi = nullptr;
  void *eta_w = nullptr, *Vphys = nullptr, *delta = nullptr, *wout = nullptr;
  void* eta_ws = nullptr;    // physical working eta of the adaptive scheme's later stages (lazy)
  double* out64 = nullptr;   // conversion buffer for one member's field
  double* stage64 = nullptr; // conversion buffer for every member's field (batch calls; lazy)
  double* stage64b = nullptr; // the second field's buffer (streamed step; lazy)
  int* d_active = nullptr;   // per-member flags for single-member passes
  int* d_conv = nullptr;     // adaptive order: 1 while a member still iterates
  int* d_orders = nullptr;   // adaptive order: orders used by the last diagnostic
  int* d_notconv = nullptr;  // adaptive order: tolerance not met at the highest order
  double* d_red = nullptr;   // adaptive order: partial norms
  double* wm_prof = nullptr; // wavemaker bells [J][nx] (FP64)
  void* wm_pg = nullptr;     // wavemaker pressure profile of the current stage (nx)
  int wm_cap = 0;            // components wm_prof has room for
  std::vector<DynTable> dyn; // h-dependent propagator tables (adaptive scheme)
  double* d_norm45 = nullptr; // adaptive scheme: per member |e_eta|^2, |e_phi|^2, |eta|^2, |phi|^2
  double* d_part45 = nullptr; // its block partials
  double* d_implicit = nullptr; // implicit form: per iteration and member |V_new - V_old|^2, |V_new|^2 (lazy)
  double* d_crest = nullptr;    // crest position and height of one member (lazy)
  std::map<std::string, void*> mixed;
  std::map<std::string, void*> tables;   // multiplier tables by key
  size_t phys_elems() const { return (size_t)nx * ny; }
  size_t mixed_elems() const { return (size_t)ny * W; }
};

// One branch of a step schedule is a Unit (schedule.h): the members [m0, m1)
// (local indices) of one group.  Every pass of a step covers whole rows and
// columns of each member, so a group's passes restricted to a member range are
// the same launches over fewer rows or columns, with the same arithmetic per
// member.

struct GraphEntry {
  double dt;
  bool prof;
  int kind = 0;                      // StepKind
  int group = -1;                    // -1: every unit of the schedule; else the members
  int m0 = 0, m1 = 0;                //   [m0, m1) of that group alone (the streamed step)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  std::vector<cudaEvent_t> ev;       // profiled graphs: event pair per pass
  std::vector<int> ev_family;
};

// What a captured graph runs: a whole step of a fixed-step scheme; or, for
// the adaptive integrating factor, its six stages with the order-5 offsets
// and the step's error norms (A), then the acceptance of the step (B).
enum StepKind { SK_STEP = 0, SK_RK45_A = 1, SK_RK45_B = 2 };


}  // namespace

struct sbi_ctx {
  std::string err = "no error";
  sbi_options opt;
  double gravity = 9.81;
  bool fp64 = false;
  bool state_ds = true;   // the state and RK sums are double-single pairs (FP32 path default)
  size_t real_size = 4;
  int nmembers = 0;
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t cap = nullptr;     // internal stream for graph capture
  std::vector<cudaStream_t> gstreams;  // one capture branch per unit of the schedule
  std::vector<cudaEvent_t> gevents;    // fork / join events of the branches
  std::vector<cudaStream_t> pstreams;  // streamed step: one stream per unit, by falling priority
  std::vector<cudaEvent_t> pevents;    // streamed step: start, then one per unit
  std::vector<Group> groups;
  std::vector<std::pair<int, int>> where;  // member -> (group, local index)
  // step schedule: the branches of a step graph (concurrent, or one after
  // another when serial), chosen by timing on the first step (choose_schedule)
  std::vector<Unit> units;
  bool serial = false;
  bool sched_done = false;
  std::string sched_report;
  int stream_k = 0;   // streamed step: each schedule unit cut into stream_k member ranges (0: not chosen)
  int stall_tx = 0;   // test hook of the staged column pass (sbi_test_stall_staged_copies)
  std::vector<void*> allocs;
  void* tw = nullptr;
  void* wgt = nullptr;  // shared sponge weight (working precision) or null
  int* d_flags = nullptr;  // [0]: non-finite state; [1]: a bounded wait gave up
  double* d_partials = nullptr;
  size_t partial_cap = 0;
  std::list<GraphEntry> graphs;   // stable addresses: two graphs may be held at once
  // profiling
  bool prof = false;
  std::vector<double> prof_ms;
  std::vector<long long> prof_launches;
  std::vector<int> orders_used;
  // autotuner: block shape per pass signature (rows or columns per block)
  struct Tuned {
    int choice, deflt;
    double ms;
  };
  std::map<std::string, Tuned> tuned;
  std::vector<std::string> tune_order;  // signatures in the order they were tuned
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  double dyn_h = NAN;   // the step the dynamic tables were last computed for
  // simulation time (advanced by sbi_step) and the pneumatic wavemaker
  double t_host = 0.0;
  double* d_time = nullptr;
  int wm_n = 0;
  double* wm_params = nullptr;  // [omega_0..omega_{J-1}, theta_0..theta_{J-1}] on the device
  int wm_params_cap = 0;
  bool filter_on() const { return opt.filt_beta1 > 0.0; }
};

namespace {

int fail(sbi_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(sbi_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SBI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                               \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

void* dalloc(sbi_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->opt.dev_alloc) {
    p = c->opt.dev_alloc(bytes, c->opt.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->allocs.push_back(p);
    cudaMemsetAsync(p, 0, bytes, c->cap);
  }
  return p;
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
// a step scalar as a double and as a double-single float pair
RkScalar rk_scalar(double v) {
  RkScalar r;
  r.d = v;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

struct Planner {
  sbi_ctx* c;
  Group& g;
  bool oom = false;      // an allocation failed (or a descriptor would overflow)
  // stage of an integrating-factor step (1..4; 0 otherwise): the diagnostic
  // then reads the stage state from st_eta / st_phi and its last order writes
  // the nonlinear part V - V_1 under a per-stage name; the dynamic condition
  // drops -g eta
  int if_stage = 0;
  std::string st_eta = "eta_m", st_phi = "phi_m";
  // the physical working eta the row passes read (nullptr: g.eta_w); the
  // adaptive scheme's stages 2..6 use their own, so that a rejected attempt
  // leaves u_n's copy intact
  void* st_eta_w = nullptr;
  void* stage_eta_w() {
    if (!g.eta_ws) {
      g.eta_ws = dalloc(c, g.phys_elems() * g.n * c->real_size);
      if (!g.eta_ws) oom = true;
    }
    return g.eta_ws;
  }

  size_t vsize() const { return 2 * c->real_size; }

  void* mixed(const std::string& name) {
    auto it = g.mixed.find(name);
    if (it != g.mixed.end()) return it->second;
    void* p = dalloc(c, g.mixed_elems() * g.n * vsize());
    if (!p) oom = true;
    g.mixed[name] = p;
    return p;
  }
  BufRef mref(const std::string& name) { return BufRef{mixed(name), (long long)g.mixed_elems()}; }
  BufRef pref(void* p, bool shared = false) {
    return BufRef{p, shared ? 0LL : (long long)g.phys_elems()};
  }
  BufRef dref(double* p) { return BufRef{p, (long long)g.phys_elems()}; }
  double mixed_bytes() const { return (double)g.mixed_elems() * g.n * vsize(); }
  double phys_bytes() const { return (double)g.phys_elems() * g.n * c->real_size; }
  double phys64_bytes() const { return (double)g.phys_elems() * g.n * 8.0; }

  // --- row pass builder ---
  struct RowB {
    RowParams p;
    int nbuf = 0;
    double bytes = 0;
    int maxslot = -1;
  };
  RowB row_begin() {
    RowB r;
    std::memset(&r.p, 0, sizeof(r.p));
    r.p.rows_total = g.n * g.ny;
    r.p.ny = g.ny;
    r.p.W = g.W;
    r.p.tw = c->tw;
    return r;
  }
  int add_buf(RowB& r, BufRef b) {
    if (r.nbuf >= kMaxRowBufs) {
      oom = true;
      return 0;
    }
    r.p.buf[r.nbuf] = b;
    return r.nbuf++;
  }
  bool room(RowB& r) {
    if (r.p.nops >= kMaxRowOps) {
      oom = true;
      return false;
    }
    return true;
  }
  void c2r(RowB& r, int slot, const std::vector<std::string>& srcs, void* phys_out = nullptr) {
    RowOp op{};
    op.kind = ROP_C2R;
    op.slot = (uint8_t)slot;
    op.a = (uint8_t)r.nbuf;
    op.b = (uint8_t)srcs.size();
    for (auto& s : srcs) add_buf(r, mref(s));
    r.bytes += mixed_bytes() * srcs.size();
    op.dst = kNone;
    if (phys_out) {
      op.dst = (uint8_t)add_buf(r, pref(phys_out));
      r.bytes += phys_bytes();
    }
    if (room(r)) r.p.ops[r.p.nops++] = op;
    r.maxslot = std::max(r.maxslot, slot);
  }
  void prod(RowB& r, int slot, int ea, int db, int wc, double coef, const std::string& dst) {
    RowOp op{};
    op.kind = ROP_PROD;
    op.slot = slot < 0 ? kNone : (uint8_t)slot;
    op.a = (uint8_t)ea;
    op.b = (uint8_t)db;
    op.c = (uint8_t)wc;
    op.coef = coef;
    op.dst = (uint8_t)add_buf(r, mref(dst));
    r.bytes += mixed_bytes();
    if (room(r)) r.p.ops[r.p.nops++] = op;
  }
  void n2(RowB& r, int slot0, const std::string& dst) {
    RowOp op{};
    op.kind = ROP_N2;
    op.slot = (uint8_t)slot0;
    op.a = g.two_d ? 2 : 1;
    op.coef = if_stage > 0 ? 0.0 : c->gravity;   // the nonlinear part has no -g eta
    op.dst = (uint8_t)add_buf(r, mref(dst));
    r.bytes += mixed_bytes();
    if (room(r)) r.p.ops[r.p.nops++] = op;
  }
  void vfw(RowB& r, int slot0, const std::string& dst) {
    RowOp op{};
    op.kind = ROP_VFW;
    op.slot = (uint8_t)slot0;
    op.a = g.two_d ? 2 : 1;
    op.dst = (uint8_t)add_buf(r, mref(dst));
    r.bytes += mixed_bytes();
    if (room(r)) r.p.ops[r.p.nops++] = op;
  }
  void wdot(RowB& r, int slot0, void* phys_out) {
    RowOp op{};
    op.kind = ROP_WDOT;
    op.slot = (uint8_t)slot0;
    op.a = g.two_d ? 2 : 1;
    op.dst = (uint8_t)add_buf(r, pref(phys_out));
    r.bytes += phys_bytes();
    if (room(r)) r.p.ops[r.p.nops++] = op;
  }
  int rpc_for(int nslots) {
    const int r = c->fp64 ? row_rpc<double>(g.nx, g.W, nslots) : row_rpc<float>(g.nx, g.W, nslots);
    if (r <= 0) oom = true;
    return r > 0 ? r : 1;
  }
  Pass row_end(RowB& r, bool use_eta, bool use_delta, bool use_w) {
    if (use_eta) {
      r.p.eta = pref(st_eta_w ? st_eta_w : g.eta_w);
      r.bytes += phys_bytes();
    }
    if (use_delta && g.variable) {
      r.p.delta = pref(g.delta);
      r.bytes += phys_bytes();
    }
    if (use_w && c->wgt) {
      r.p.wgt = pref(c->wgt, true);
      r.bytes += (double)g.phys_elems() * c->real_size;
    }
    r.p.nslots = r.maxslot + 1;
    r.p.rpc = rpc_for(r.p.nslots);
    Pass ps{};
    ps.kind = PK_ROW;
    ps.nsize = g.nx;
    ps.row = r.p;
    ps.bytes = r.bytes;
    int nx_fields = 0;  // every op but WDOT transforms one field along x
    for (int o = 0; o < r.p.nops; ++o) nx_fields += r.p.ops[o].kind != ROP_WDOT;
    ps.xforms = (double)nx_fields * g.phys_elems() * g.n;
    return ps;
  }

  // --- column pass builder ---
  struct ColIn {
    std::string name;
    std::vector<ColTerm> terms;
  };
  static ColTerm term(int acc, double cc, int kpow, int depth, int gx, int gy, int mask = 0) {
    ColTerm t{};
    t.acc = (uint8_t)acc;
    t.c = cc;
    t.kpow = (int8_t)kpow;
    t.depth = (uint8_t)depth;
    t.gx = (uint8_t)gx;
    t.gy = (uint8_t)gy;
    t.mask = (uint8_t)mask;
    return t;
  }
  // Device table of a multiplier (created once per group and key).
  const void* table(const ColTerm& t) {
    char key[160];
    // dynamic tables (pad_ = 1 + p) depend on the step h: tau = r h with the
    // ratio r in t.tau, coefficient t.c h^p; their values are written by
    // update_dyn_tables whenever h changes
    const bool dyn = t.pad_ != 0;
    snprintf(key, sizeof(key), "%s%.17g|%d|%d|%d|%d|%d|%.17g", dyn ? (t.pad_ == 2 ? "h1|" : "h0|") : "",
             t.c, t.kpow, t.depth, t.gx, t.gy, t.mask, (dyn || t.depth >= 4) ? t.tau : 0.0);
    auto it = g.tables.find(key);
    if (it != g.tables.end()) return it->second;
    void* p = dalloc(c, (size_t)g.W * g.ny * c->real_size);
    if (!p) {
      oom = true;
      return nullptr;
    }
    TableSpec s{};
    s.W = g.W;
    s.ny = g.ny;
    s.kx_keep = g.kx_keep;
    s.ky_keep = g.ky_keep;
    s.two_pi_over_Lx = 2.0 * M_PI / g.Lx;
    s.two_pi_over_Ly = g.two_d ? 2.0 * M_PI / g.Ly : 0.0;
    s.h0 = g.deep ? INFINITY : g.h0;
    s.filt_kf = c->filter_on() ? c->opt.filt_beta1 * c->opt.k_ref : 0.0;
    s.filt_beta2 = c->opt.filt_beta2;
    s.c = t.c;
    s.tau = t.tau;
    s.gravity = c->gravity;
    s.kpow = t.kpow;
    s.depth = t.depth;
    s.gx = t.gx;
    s.gy = t.gy;
    s.mask = t.mask;
    g.tables[key] = p;
    if (dyn) {
      g.dyn.push_back(DynTable{p, s, t.tau, t.pad_ - 1});
      c->dyn_h = NAN;   // the new table has no values yet
      return p;
    }
    cudaError_t e = c->fp64 ? launch_coef_table<double>(p, s, c->cap) : launch_coef_table<float>(p, s, c->cap);
    if (e != cudaSuccess) oom = true;
    return p;
  }

  Pass col(const std::vector<ColIn>& ins, const std::vector<std::pair<std::string, ColTerm>>& outs,
           int nacc, const std::vector<std::string>& passthrough = {}) {
    ColParams p;
    std::memset(&p, 0, sizeof(p));
    p.W = g.W;
    p.ny = g.ny;
    p.nx = g.nx;
    p.cols_total = g.n * g.W;
    p.two_pi_over_Lx = 2.0 * M_PI / g.Lx;
    p.two_pi_over_Ly = g.two_d ? 2.0 * M_PI / g.Ly : 0.0;
    p.h0 = g.deep ? INFINITY : g.h0;
    p.kx_keep = g.kx_keep;
    p.ky_keep = g.ky_keep;
    p.filt_kf = c->filter_on() ? c->opt.filt_beta1 * c->opt.k_ref : 0.0;
    p.filt_beta2 = c->opt.filt_beta2;
    p.nacc = nacc;
    p.tw = c->tw;
    p.err_flag = c->d_flags + 1;
    p.stall_tx = c->stall_tx;
    p.staged = (c->opt.col_staging == 1 &&
                (c->fp64 ? col_stageable<double>(g.ny) : col_stageable<float>(g.ny))) ? 1 : 0;
    const double scale = 1.0 / ((double)g.nx * g.ny);
    size_t total_terms = 0;
    for (auto& in : ins) total_terms += in.terms.size();
    if (ins.size() + outs.size() > (size_t)kMaxColBufs || total_terms > (size_t)kMaxColTerms ||
        outs.size() > (size_t)kMaxColOuts || nacc > kMaxColAcc) {
      oom = true;
      Pass ps{};
      ps.kind = PK_COL;
      return ps;
    }
    int nt = 0;
    for (size_t i = 0; i < ins.size(); ++i) {
      p.buf[i] = mref(ins[i].name);
      p.term_begin[i] = nt;
      for (auto t : ins[i].terms) {
        t.in = (uint8_t)i;
        t.c *= scale;
        t.tab = table(t);
        p.terms[nt++] = t;
      }
    }
    p.nin = (int)ins.size();
    p.term_begin[p.nin] = nt;
    p.nterms = nt;
    for (size_t o = 0; o < outs.size(); ++o) {
      ColTerm t = outs[o].second;
      t.in = (uint8_t)(p.nin + o);
      t.tab = table(t);
      p.buf[p.nin + o] = mref(outs[o].first);
      p.outs[o] = t;
    }
    p.nouts = (int)outs.size();
    if (passthrough.size() > 8) {
      oom = true;
    } else {
      for (size_t q = 0; q < passthrough.size(); ++q) p.pass[q] = mref(passthrough[q]);
      p.npass = (int)passthrough.size();
    }
    Pass ps{};
    ps.kind = PK_COL;
    ps.nsize = g.ny;
    ps.col = p;
    ps.bytes = mixed_bytes() * (ins.size() + outs.size() + passthrough.size());
    // every input and output is one field transformed along y
    ps.xforms = g.ny > 1 ? (double)(ins.size() + outs.size()) * g.phys_elems() * g.n : 0.0;
    return ps;
  }

  std::vector<char> dims() const { return g.two_d ? std::vector<char>{'x', 'y'} : std::vector<char>{'x'}; }
  static std::string S(const char* f, int a) { char b[64]; snprintf(b, 64, f, a); return b; }
  static std::string S2(const char* f, int a, int b2) { char b[64]; snprintf(b, 64, f, a, b2); return b; }

  static double fact(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

  // Col A: order 1 (Sec. 2.4) and the gradients of phi~ and eta.
  Pass plan_col_a() {
    const bool var = g.variable;
    std::vector<ColIn> ins = {{st_phi, {term(0, 1.0, 0, 0, 0, 0)}},
                              {st_eta, {term(1, 1.0, 0, 0, 0, 0)}}};
    std::vector<std::pair<std::string, ColTerm>> outs;
    outs.push_back({"V1", term(0, 1.0, 1, 1, 0, 0, 1)});  // k tanh(kh) phi^
    for (char d : dims()) {
      const int gx = d == 'x', gy = d == 'y';
      outs.push_back({std::string("dphi") + d, term(0, 1.0, 0, 0, gx, gy, 1)});
      outs.push_back({std::string("deta") + d, term(1, 1.0, 0, 0, gx, gy, 1)});
      if (var) outs.push_back({std::string("db1") + d, term(0, 1.0, 0, 2, gx, gy, 1)});  // ik sech phi^
    }
    return col(ins, outs, 2);
  }

  // Row l: eager products of order l-1 (see file header), formed as running
  // products (the slot is multiplied by eta or delta once per product).
  Pass plan_row_level(int l) {
    const int M = c->opt.order;
    RowB r = row_begin();
    c2r(r, 0, {S("V%d", l - 1)});
    for (int j = 1; j <= M - (l - 1); ++j) prod(r, 0, 1, 0, 2, 1.0, S2("P%d_%d", j, l - 1));
    if (l == 2) {
      for (char d : dims()) {
        c2r(r, 0, {std::string("dphi") + d});
        for (int j = 1; j <= M - 1; ++j) prod(r, 0, 1, 0, 2, 1.0, S("Q%d", j) + d);
      }
    }
    bool use_delta = false;
    if (g.variable && l - 1 <= M - 1) {
      const int m = l - 1;
      for (char d : dims()) {
        c2r(r, 0, {S("db%d", m) + d});
        int jprev = 0;
        for (int j = 1; j <= M - m; ++j) {
          const int ll = j + m;
          if (ll <= M - 1 || (j % 2 == 1)) {
            prod(r, 0, 0, j - jprev, 2, 1.0, S2("R%d_%d", j, m) + d);
            jprev = j;
            use_delta = true;
          }
        }
      }
    }
    return row_end(r, true, use_delta, false);
  }

  // Col l: F{V_l} (acc 0) and F{varphi_l} (acc 1) of Appendix C:
  //  F{V_l}   = sum_j -k^j/j! T_j F{eta^j V_{l-j}} - T_l k^{l-2}/(l-1)! ik.F{eta^{l-1} grad phi~}
  //             + sum_{j odd} k^{j-1}/j! sech ik.F{delta^j grad varphi_{l-j}}
  //  F{varphi_l} = sum_{j odd} -k^{j-1}/j! sech F{eta^j V_{l-j}}
  //             - [l odd] sech k^{l-3}/(l-1)! ik.F{eta^{l-1} grad phi~}
  //             + sum_j (-1)^j k^{j-2}/j! T_j ik.F{delta^j grad varphi_{l-j}}
  // with T_j = tanh(kh) for odd j and 1 for even j.
  Pass plan_col_level(int l) {
    const int M = c->opt.order;
    const bool phi_out = g.variable && l <= M - 1;
    std::vector<ColIn> ins;
    for (int j = 1; j < l; ++j) {
      ColIn in{S2("P%d_%d", j, l - j), {}};
      in.terms.push_back(term(0, -1.0 / fact(j), j, (j % 2) ? 1 : 0, 0, 0));
      if (phi_out && (j % 2 == 1)) in.terms.push_back(term(1, -1.0 / fact(j), j - 1, 2, 0, 0));
      ins.push_back(in);
    }
    for (char d : dims()) {
      const int gx = d == 'x', gy = d == 'y';
      ColIn in{S("Q%d", l - 1) + d, {}};
      in.terms.push_back(term(0, -1.0 / fact(l - 1), l - 2, (l % 2) ? 1 : 0, gx, gy));
      if (phi_out && (l % 2 == 1)) in.terms.push_back(term(1, -1.0 / fact(l - 1), l - 3, 2, gx, gy));
      ins.push_back(in);
    }
    if (g.variable) {
      for (int j = 1; j < l; ++j) {
        const bool to_v = (j % 2 == 1);
        if (!to_v && !phi_out) continue;
        for (char d : dims()) {
          const int gx = d == 'x', gy = d == 'y';
          ColIn in{S2("R%d_%d", j, l - j) + d, {}};
          if (to_v) in.terms.push_back(term(0, 1.0 / fact(j), j - 1, 2, gx, gy));
          if (phi_out) {
            if (j == 1) in.terms.push_back(term(1, -1.0, -1, 1, gx, gy));
            else if (j % 2) in.terms.push_back(term(1, -1.0 / fact(j), j - 2, 1, gx, gy));
            else in.terms.push_back(term(1, 1.0 / fact(j), j - 2, 0, gx, gy));
          }
          ins.push_back(in);
        }
      }
    }
    std::vector<std::pair<std::string, ColTerm>> outs;
    // the last order is written as the sum V^_1 + ... + V^_M (mixed), the only
    // form in which it is used
    const bool last = l == M;
    outs.push_back({last ? (if_stage > 0 ? S("Vnl%d", if_stage) : std::string("Vsum")) : S("V%d", l),
                    term(0, 1.0, 0, 0, 0, 0, 1)});
    if (phi_out) {
      for (char d : dims())
        outs.push_back({S("db%d", l) + d, term(1, 1.0, 0, 0, d == 'x', d == 'y', 1)});
    }
    std::vector<std::string> pass;
    if (last)   // the integrating-factor stages leave out V_1 (the linear part)
      for (int q = if_stage > 0 ? 2 : 1; q < M; ++q) pass.push_back(S("V%d", q));
    return col(ins, outs, phi_out ? 2 : 1, pass);
  }

  // mixed buffers whose sum is F_x{V}
  std::vector<std::string> v_names() const {
    const bool hos = c->opt.diagnostic == SBI_DIAG_HOS;
    if (c->opt.order == 1 && !hos) return {std::string("V1")};
    if (if_stage > 0) return {S("Vnl%d", if_stage), std::string("V1")};
    return {std::string("Vsum")};
  }

  Pass plan_conv(int phase, int l) {
    Pass ps{};
    ps.kind = PK_CONV;
    ConvParams& q = ps.conv;
    q.phase = phase;
    // the highest order exists only inside the sum Vsum: there the increment is
    // Vsum - (V_1 + .. + V_{M-1}), read from the M - 1 lower-order buffers
    q.nlev = (l == c->opt.order) ? l - 1 : l;
    for (int m = 1; m <= q.nlev && m <= 7; ++m) q.V[m - 1] = mixed(S("V%d", m));
    q.vsum = mixed("Vsum");
    q.stride = (long long)g.mixed_elems();
    q.W = g.W;
    q.ny = g.ny;
    q.n = g.n;
    q.level = l;
    q.last = l == c->opt.order;
    q.tol2 = c->opt.adapt_tol * c->opt.adapt_tol;
    q.conv = g.d_conv;
    q.orders = g.d_orders;
    q.notconv = g.d_notconv;
    q.red = g.d_red;
    ps.bytes = phase == 1 ? mixed_bytes() * l : (phase == 2 ? mixed_bytes() * (l + 1) : 0.0);
    return ps;
  }

  // HOS diagnostic (flat bottom), the perturbation expansion of the section
  // comparing ESBI and HOS: d^n/dz^n at z = 0 multiplies mode k by k^n T_n
  // (T_n = tanh(k h0) for odd n, 1 for even n).
  //   phi^(1) = phi~,  phi^(m) = -sum_{n=1}^{m-1} eta^n/n! d^n_z phi^(m-n),
  //   W = sum_{n=0}^{M-1} eta^n/n! sum_{m=1}^{M-n} d^{n+1}_z phi^(m),
  //   V = W (1 + |grad eta|^2) - grad eta . grad phi~,
  // every phi^(m), W and V dealiased.  Column passes turn each order into its
  // z-derivatives HD<m>_<n> (mixed); row passes form the products.
  void plan_hos_diag(std::vector<Pass>& out) {
    const int M = c->opt.order;
    auto dz = [&](int n) { return term(0, 1.0, n, (n % 2) ? 1 : 0, 0, 0, 1); };
    {
      std::vector<ColIn> ins = {{st_phi, {term(0, 1.0, 0, 0, 0, 0)}},
                                {st_eta, {term(1, 1.0, 0, 0, 0, 0)}}};
      std::vector<std::pair<std::string, ColTerm>> outs;
      for (int n = 1; n <= M; ++n) outs.push_back({S2("HD%d_%d", 1, n), dz(n)});
      for (char d : dims()) {
        const int gx = d == 'x', gy = d == 'y';
        outs.push_back({std::string("dphi") + d, term(0, 1.0, 0, 0, gx, gy, 1)});
        outs.push_back({std::string("deta") + d, term(1, 1.0, 0, 0, gx, gy, 1)});
      }
      out.push_back(col(ins, outs, 2));
    }
    for (int m = 2; m <= M; ++m) {
      RowB r = row_begin();
      for (int n = 1; n < m; ++n) {
        c2r(r, 0, {S2("HD%d_%d", m - n, n)});
        prod(r, 0, n, 0, 0, -1.0 / fact(n), S2("HP%d_%d", m, n));
      }
      out.push_back(row_end(r, true, false, false));
      std::vector<ColIn> ins;
      for (int n = 1; n < m; ++n) ins.push_back({S2("HP%d_%d", m, n), {term(0, 1.0, 0, 0, 0, 0)}});
      std::vector<std::pair<std::string, ColTerm>> outs;
      for (int n = 1; n <= M - m + 1; ++n) outs.push_back({S2("HD%d_%d", m, n), dz(n)});
      out.push_back(col(ins, outs, 1));
    }
    {
      RowB r = row_begin();
      for (int n = 0; n < M; ++n) {
        std::vector<std::string> src;
        for (int m = 1; m <= M - n; ++m) src.push_back(S2("HD%d_%d", m, n + 1));
        c2r(r, 0, src);
        prod(r, 0, n, 0, 0, 1.0 / fact(n), S("HW%d", n));
      }
      out.push_back(row_end(r, true, false, false));
      std::vector<ColIn> ins;
      for (int n = 0; n < M; ++n) ins.push_back({S("HW%d", n), {term(0, 1.0, 0, 0, 0, 0)}});
      out.push_back(col(ins, {{"HWs", term(0, 1.0, 0, 0, 0, 0, 1)}}, 1));
    }
    {
      RowB r = row_begin();
      c2r(r, 0, {"HWs"});
      int s = 1;
      for (char d : dims()) c2r(r, s++, {std::string("deta") + d});
      for (char d : dims()) c2r(r, s++, {std::string("dphi") + d});
      vfw(r, 0, "HVr");
      out.push_back(row_end(r, false, false, false));
      if (if_stage > 0) {
        // integrating factor: the nonlinear part V - k tanh(kh) phi^ and V_1
        std::vector<ColIn> ins = {{"HVr", {term(0, 1.0, 0, 0, 0, 0)}},
                                  {st_phi, {term(0, -1.0, 1, 1, 0, 0), term(1, 1.0, 1, 1, 0, 0)}}};
        out.push_back(col(ins, {{S("Vnl%d", if_stage), term(0, 1.0, 0, 0, 0, 0, 1)},
                                {"V1", term(1, 1.0, 0, 0, 0, 0, 1)}}, 2));
      } else {
        out.push_back(col({{"HVr", {term(0, 1.0, 0, 0, 0, 0)}}}, {{"Vsum", term(0, 1.0, 0, 0, 0, 0, 1)}}, 1));
      }
    }
  }

  void plan_diag(std::vector<Pass>& out) {
    if (c->opt.diagnostic == SBI_DIAG_HOS) {
      plan_hos_diag(out);
      return;
    }
    const bool adapt = c->opt.adapt_tol > 0.0 && c->opt.order > 1;
    if (adapt) out.push_back(plan_conv(0, 1));
    out.push_back(plan_col_a());
    for (int l = 2; l <= c->opt.order; ++l) {
      Pass r = plan_row_level(l), q = plan_col_level(l);
      if (adapt) {
        r.row.active = g.d_conv;
        q.col.active = g.d_conv;
      }
      out.push_back(r);
      out.push_back(q);
      if (adapt) {
        if (l < c->opt.order) {
          out.push_back(plan_conv(1, l));
          out.push_back(plan_conv(2, l));
        } else {
          out.push_back(plan_conv(1, l));
        }
        out.push_back(plan_conv(3, l));
      }
    }
  }

  // Row RHS + Col RHS: phi~_t = M F^{-1}{F{N2} + nu ik/k^2 . F{w grad phi~}}
  void plan_rhs(std::vector<Pass>& out, double stage_offset = 0.0) {
    if (c->wm_n > 0) {
      Pass w{};
      w.kind = PK_WMK;
      w.nsize = g.nx;
      w.wmk = WmkParams{g.wm_prof, c->wm_params, c->wm_params + c->wm_n, c->d_time, stage_offset,
                        g.wm_pg, c->wm_n, g.nx};
      w.bytes = (double)c->wm_n * g.nx * 8 + (double)g.nx * c->real_size;
      out.push_back(w);
    }
    RowB r = row_begin();
    c2r(r, 0, v_names(), g.Vphys);
    int s = 1;
    for (char d : dims()) c2r(r, s++, {std::string("deta") + d});
    const int sphi = s;
    for (char d : dims()) c2r(r, s++, {std::string("dphi") + d});
    n2(r, 0, "N2");
    const bool sponge = c->wgt != nullptr && c->opt.sponge_nu != 0.0;
    if (sponge) {
      int q = sphi;
      for (char d : dims()) prod(r, q++, 0, 0, 1, 1.0, std::string("SP") + d);
    }
    out.push_back(row_end(r, true, false, sponge));
    if (c->wm_n > 0) out.back().row.pg = g.wm_pg;
    std::vector<ColIn> ins = {{"N2", {term(0, 1.0, 0, 0, 0, 0)}}};
    if (sponge) {
      for (char d : dims())
        ins.push_back({std::string("SP") + d,
                       {term(0, c->opt.sponge_nu, -2, 0, d == 'x', d == 'y')}});
    }
    out.push_back(col(ins, {{if_stage > 0 ? S("phit%d", if_stage) : std::string("phit"),
                             term(0, 1.0, 0, 0, 0, 0, 1)}}, 1));
  }

  // cor_eta / cor_phi: the mixed corrections of RK_CORRECT / RK_OFFSET;
  // w_eta / w_phi: where the tail writes the mixed working copies
  Pass plan_rk(int mode, int stage, double dt, int tail, const char* cor_eta = "Ce",
               const char* cor_phi = "Cp", const char* w_eta = "eta_m", const char* w_phi = "phi_m",
               void* w_phys = nullptr) {
    RkParams p;
    std::memset(&p, 0, sizeof(p));
    p.mode = mode;
    p.stage = stage;
    p.tail = tail;
    p.rows_total = g.n * g.ny;
    p.ny = g.ny;
    p.W = g.W;
    {
      const int tpr = c->fp64 ? row_tpr<double>(g.nx) : row_tpr<float>(g.nx);
      p.rpc = std::max(1, kRkThreads / std::max(1, tpr));
    }
    p.dt = dt;
    p.state64 = c->fp64 || !c->state_ds;
    p.dt6 = rk_scalar(dt / 6.0);
    p.cdt = rk_scalar((stage == 3 ? 1.0 : 0.5) * dt);
    p.eta0 = dref(g.eta0);
    p.phi0 = dref(g.phi0);
    p.acc_eta = dref(g.acc_eta);
    p.acc_phi = dref(g.acc_phi);
    p.V = pref(g.Vphys);
    const bool corr = mode == RK_CORRECT || mode == RK_OFFSET;
    p.phit = mref(corr ? cor_eta : "phit");
    p.corr_phi = mref(cor_phi);
    p.eta_w = pref(w_phys ? w_phys : g.eta_w);
    p.eta_hat = mref(w_eta);
    p.phi_hat = mref(w_phi);
    p.nonfinite = c->d_flags;
    p.tw = c->tw;
    // transforms along x: the stage's phi~_t (STAGE) or the two corrections
    // (CORRECT) back to physical space, and the working copies forward (tail)
    const int nxf = (mode == RK_STAGE ? 1 : (corr ? 2 : 0)) + (tail ? 2 : 0);
    const double xforms = (double)nxf * g.phys_elems() * g.n;
    double b = phys64_bytes() * 2;  // read master
    if (mode == RK_STAGE) {
      b += mixed_bytes() + phys_bytes();                      // phi~_t, V
      b += phys64_bytes() * 2 * ((stage > 1 ? 1 : 0) + (stage < 4 ? 1 : 0));  // sums
      if (stage == 4) b += phys64_bytes() * 2;                 // write master
    } else if (mode == RK_CORRECT) {
      b += mixed_bytes() * 2 + phys64_bytes() * 2;
    } else if (mode == RK_OFFSET) {
      b += mixed_bytes() * 2;
    }
    if (tail) b += phys_bytes() + 2 * mixed_bytes();
    Pass ps{};
    ps.kind = PK_RK;
    ps.nsize = g.nx;
    ps.rk = p;
    ps.bytes = b;
    ps.xforms = xforms;
    return ps;
  }

  // (M Lambda - 1) correction of the FP64 state, applied through RK_CORRECT.
  // entry = false: the pass before already wrote the state's working copies
  // (eta_m, phi_m) with its tail.
  void plan_project(std::vector<Pass>& out, bool with_filter, bool entry = true) {
    if (entry) out.push_back(plan_rk(RK_ENTRY, 0, 0.0, 1));
    const int depth = with_filter ? 3 : 0;
    out.push_back(col({{"eta_m", {term(0, 1.0, 0, 0, 0, 0)}}, {"phi_m", {term(1, 1.0, 0, 0, 0, 0)}}},
                      {{"Ce", term(0, 1.0, 0, depth, 0, 0, 2)}, {"Cp", term(1, 1.0, 0, depth, 0, 0, 2)}},
                      2));
    out.push_back(plan_rk(RK_CORRECT, 0, 0.0, 1));
  }

  // Integrating-factor (Lawson) combination after the right-hand side of stage
  // s: with E(tau) = e^{A tau} (propagator tables), u_n = (eta_m, phi_m) and
  // k_s = (Vnl<s>, phit<s>), the mixed offsets (De, Dp) from u_n of
  //   s = 1: (E(h/2) - I) u_n + h/2 E(h/2) k1          (stage 2 state)
  //   s = 2: (E(h/2) - I) u_n + h/2 k2                 (stage 3 state)
  //   s = 3: (E(h) - I) u_n + h E(h/2) k3              (stage 4 state)
  //   s = 4: (E(h) - I) u_n + h/6 (E(h) k1 + 2 E(h/2)(k2 + k3) + k4)   (u_{n+1})
  // u_n's working spectra come from a row transform (unnormalised in x, like
  // every column-pass input) while the k_s are column-pass outputs, normalised
  // for the inverse row transform: their coefficients carry the factor nx.
  Pass plan_if_combine(int s, double h) {
    std::map<std::string, std::vector<ColTerm>> terms;
    std::vector<std::string> order;
    auto add = [&](const std::string& name, ColTerm t) {
      if (!terms.count(name)) order.push_back(name);
      terms[name].push_back(t);
    };
    auto prop = [&](int acc, double cc, int depth, double tau) {
      ColTerm t = term(acc, cc, 0, depth, 0, 0);
      t.tau = tau;
      return t;
    };
    // (E(tau) - I) applied to the state's pair (a, b)
    auto apply_E_minus_I = [&](const std::string& a, const std::string& b, double tau) {
      add(a, prop(0, 1.0, 4, tau));
      add(a, prop(1, -1.0, 6, tau));
      add(b, prop(0, 1.0, 5, tau));
      add(b, prop(1, 1.0, 4, tau));
    };
    // order 1 of the successive approximation: V - V_1 = 0 (not so for HOS)
    const bool has_vnl = c->opt.order > 1 || c->opt.diagnostic == SBI_DIAG_HOS;
    const double nrm = (double)g.nx;
    // cc E(tau) k_q (prop_it) or cc k_q
    auto k_pair = [&](int q, double cc, double tau, bool prop_it) {
      const std::string ke = S("Vnl%d", q), kp = S("phit%d", q);
      cc *= nrm;
      if (prop_it) {
        if (has_vnl) {
          add(ke, prop(0, cc, 7, tau));
          add(ke, prop(1, -cc, 6, tau));
        }
        add(kp, prop(0, cc, 5, tau));
        add(kp, prop(1, cc, 7, tau));
      } else {
        if (has_vnl) add(ke, term(0, cc, 0, 0, 0, 0));
        add(kp, term(1, cc, 0, 0, 0, 0));
      }
    };
    const double half = 0.5 * h;
    if (s == 1) {
      apply_E_minus_I("eta_m", "phi_m", half);
      k_pair(1, half, half, true);
    } else if (s == 2) {
      apply_E_minus_I("eta_m", "phi_m", half);
      k_pair(2, half, 0.0, false);
    } else if (s == 3) {
      apply_E_minus_I("eta_m", "phi_m", h);
      k_pair(3, h, half, true);
    } else {
      apply_E_minus_I("eta_m", "phi_m", h);
      k_pair(1, h / 6.0, h, true);
      k_pair(2, h / 3.0, half, true);
      k_pair(3, h / 3.0, half, true);
      k_pair(4, h / 6.0, 0.0, false);
    }
    std::vector<ColIn> ins;
    for (const auto& name : order) ins.push_back({name, terms[name]});
    return col(ins, {{"De", term(0, 1.0, 0, 0, 0, 0, 1)}, {"Dp", term(1, 1.0, 0, 0, 0, 0, 1)}}, 2);
  }

  // Adaptive integrating factor, Cash-Karp 5(4) pair: mixed offsets from u_n
  // (eta_m, phi_m) with the stored k_j = (Vnl<j>, phit<j>) (nx-normalised
  // like in plan_if_combine), E(tau) from h-dependent tables:
  //   target 2..6: stage state  (E(c_i h) - I) u_n + h sum_j a_ij E((c_i - c_j) h) k_j -> (De, Dp)
  //   target 7:    order 5      (E(h) - I) u_n + h sum_j b5_j E((1 - c_j) h) k_j      -> (De, Dp)
  //   target 8:    error        h sum_j (b5_j - b4_j) E((1 - c_j) h) k_j            -> (Ee, Ep)
  Pass plan_ck_combine(int target) {
    std::map<std::string, std::vector<ColTerm>> terms;
    std::vector<std::string> order;
    auto add = [&](const std::string& name, ColTerm t) {
      if (!terms.count(name)) order.push_back(name);
      terms[name].push_back(t);
    };
    auto dyn = [&](int acc, double cc, int depth, double r, int p) {
      ColTerm t = term(acc, cc, 0, depth, 0, 0);
      t.tau = r;
      t.pad_ = (uint8_t)(1 + p);
      return t;
    };
    const double ci = target <= 6 ? kCkC[target - 1] : 1.0;
    if (target <= 7) {
      add("eta_m", dyn(0, 1.0, 4, ci, 0));
      add("eta_m", dyn(1, -1.0, 6, ci, 0));
      add("phi_m", dyn(0, 1.0, 5, ci, 0));
      add("phi_m", dyn(1, 1.0, 4, ci, 0));
    }
    const bool has_vnl = c->opt.order > 1 || c->opt.diagnostic == SBI_DIAG_HOS;
    const int nj = target <= 6 ? target - 1 : 6;
    for (int j = 1; j <= nj; ++j) {
      const double w = target <= 6 ? kCkA[target - 1][j - 1]
                                   : (target == 7 ? kCkB5[j - 1] : kCkB5[j - 1] - kCkB4[j - 1]);
      if (w == 0.0) continue;
      const double r = ci - kCkC[j - 1];
      const double cc = w * g.nx;
      const std::string ke = S("Vnl%d", j), kp = S("phit%d", j);
      if (has_vnl) {
        add(ke, dyn(0, cc, 7, r, 1));
        add(ke, dyn(1, -cc, 6, r, 1));
      }
      add(kp, dyn(0, cc, 5, r, 1));
      add(kp, dyn(1, cc, 7, r, 1));
    }
    std::vector<ColIn> ins;
    for (const auto& name : order) ins.push_back({name, terms[name]});
    const bool err = target == 8;
    return col(ins, {{err ? "Ee" : "De", term(0, 1.0, 0, 0, 0, 0, 1)},
                     {err ? "Ep" : "Dp", term(1, 1.0, 0, 0, 0, 0, 1)}}, 2);
  }

  // Per-member FP64 squared norms of the error (Ee, Ep) and of u_n (eta_m,
  // phi_m) on the kept modes (Parseval weights).
  Pass plan_norm45() {
    if (!g.d_norm45) {
      g.d_norm45 = (double*)dalloc(c, (size_t)g.n * 4 * sizeof(double));
      g.d_part45 = (double*)dalloc(c, (size_t)g.n * kConvBlocks * 4 * sizeof(double));
      if (!g.d_norm45 || !g.d_part45) oom = true;
    }
    Pass ps{};
    ps.kind = PK_NORM;
    ps.nsize = g.ny;
    ps.norm = NormParams{mixed("Ee"), mixed("Ep"), mixed("eta_m"), mixed("phi_m"),
                         (long long)g.mixed_elems(), g.W, g.ny, g.n, g.d_part45, g.d_norm45};
    ps.bytes = mixed_bytes() * 4;
    return ps;
  }

  void plan_sum_v(std::vector<Pass>& out, bool eulerian) {
    RowB r = row_begin();
    c2r(r, 0, v_names(), g.Vphys);
    if (eulerian) {
      int s = 1;
      for (char d : dims()) c2r(r, s++, {std::string("deta") + d});
      for (char d : dims()) c2r(r, s++, {std::string("dphi") + d});
      wdot(r, 0, g.wout);
    }
    out.push_back(row_end(r, false, false, false));
  }

  // Implicit form of Appendix A on a flat bottom (the iteration the
  // successive scheme replaces).  Every term of V^(2..M) is
  // C_h k c F{eta^a F^{-1}{mult F{eta^b X}}}, m = a + b, X = V or (under ik.)
  // grad phi~: for X = grad phi~ with m odd, or X = V with m even,
  // c = (-1)^{a+1}/(a! b!) and mult = C_h^{-1} (a even) or D_h^{-1} (a odd)
  // times k^{m-2} (grad phi~) or k^{m-1} (V); otherwise c = 1/(a! b!) and
  // mult = e_h k^{m-2} or e_h k^{m-1}, e_h = e^{-2kh} (zero in deep water).
  // The inner spectra S_a = sum_b c mult F{eta^b X} are formed by column
  // passes (two per pass), the products eta^a F^{-1}{S_a} by a row pass and
  // the outer C_h k sum by a last column pass.  F{V} = G + L(V): G (V^(1) and
  // the grad phi~ terms) once, L(V) per iteration.
  bool implicit_term(int acc, int a, int b, bool of_v, int gx, int gy, ColTerm* t) const {
    const int m = a + b;
    if (m == 0) return false;
    const bool direct = of_v ? (m % 2 == 0) : (m % 2 == 1);
    const int kp = of_v ? m - 1 : m - 2;
    const double f = fact(a) * fact(b);
    if (direct) {
      *t = term(acc, ((a % 2) ? 1.0 : -1.0) / f, kp, (a % 2) ? 9 : 8, gx, gy, 1);
      return true;
    }
    if (g.deep) return false;
    *t = term(acc, 1.0 / f, kp, 10, gx, gy, 1);
    return true;
  }
  // Inner spectra <prefix><o>, o = 0..nout-1, two per column pass; every
  // input gives its term for output o (acc: the pass's accumulator) or none.
  // Returns which outputs have any term.
  using TermFn = std::function<bool(int o, int acc, ColTerm* t)>;
  std::vector<bool> plan_inner(std::vector<Pass>& out, int nout, const std::string& prefix,
                               const std::vector<std::pair<std::string, TermFn>>& inputs) {
    std::vector<bool> has(std::max(nout, 0), false);
    for (int o0 = 0; o0 < nout; o0 += 2) {
      std::vector<ColIn> ins;
      bool used[2] = {false, false};
      for (const auto& def : inputs) {
        ColIn in{def.first, {}};
        for (int acc = 0; acc < 2 && o0 + acc < nout; ++acc) {
          ColTerm t;
          if (def.second(o0 + acc, acc, &t)) {
            in.terms.push_back(t);
            used[acc] = true;
          }
        }
        if (!in.terms.empty()) ins.push_back(in);
      }
      if (ins.empty()) continue;
      std::vector<std::pair<std::string, ColTerm>> outs;
      for (int acc = 0; acc < 2 && o0 + acc < nout; ++acc) {
        if (!used[acc]) continue;
        has[o0 + acc] = true;
        outs.push_back({prefix + std::to_string(o0 + acc), term(acc, 1.0, 0, 0, 0, 0, 1)});
      }
      out.push_back(col(ins, outs, used[1] ? 2 : 1));
    }
    return has;
  }
  // inputs of the V equation's inner spectra S_a: F{eta^b X} (X = V, or
  // grad phi~ when phi_terms), b = 0..M-1
  std::vector<std::pair<std::string, TermFn>> inner_eta_inputs(bool of_v, const std::string& name) {
    const int M1 = c->opt.order - 1;
    std::vector<std::pair<std::string, TermFn>> v;
    const std::vector<char> ds = of_v ? std::vector<char>{'s'} : dims();
    for (int b = 0; b <= M1; ++b)
      for (char d : ds)
        v.push_back({of_v ? S(name.c_str(), b) : S(name.c_str(), b) + d,
                     [this, b, d, of_v, M1](int a, int acc, ColTerm* t) {
                       return a + b <= M1 && implicit_term(acc, a, b, of_v, d == 'x', d == 'y', t);
                     }});
    return v;
  }
  // F{eta^a F^{-1}{S_a}} (a >= 1) by one row pass: IU<a> (prefix_u)
  void plan_implicit_outer(std::vector<Pass>& out, const std::vector<bool>& has, const std::string& prefix_s,
                           const std::string& prefix_u) {
    RowB r = row_begin();
    bool any = false;
    for (size_t a = 1; a < has.size(); ++a) {
      if (!has[a]) continue;
      c2r(r, 0, {prefix_s + std::to_string(a)});
      prod(r, 0, (int)a, 0, 0, 1.0, prefix_u + std::to_string(a));
      any = true;
    }
    if (any) out.push_back(row_end(r, true, false, false));
  }
  // the outer sum C_h k (nx S_0 + sum_{a>=1} F{eta^a s_a}) (+ extra inputs),
  // written to dst with the pass-through buffers added
  void plan_implicit_sum(std::vector<Pass>& out, const std::vector<bool>& has, const std::string& prefix_s,
                         const std::string& prefix_u, std::vector<ColIn> ins, const std::string& dst,
                         const std::vector<std::string>& passthrough) {
    // S_0 is a column-pass output (x-spectrum / nx): scaled back to the
    // unnormalised input convention of the column pass
    if (!has.empty() && has[0]) ins.push_back({prefix_s + "0", {term(0, (double)g.nx, 1, 11, 0, 0)}});
    for (size_t a = 1; a < has.size(); ++a)
      if (has[a]) ins.push_back({prefix_u + std::to_string(a), {term(0, 1.0, 1, 11, 0, 0)}});
    out.push_back(col(ins, {{dst, term(0, 1.0, 0, 0, 0, 0, 1)}}, 1, passthrough));
  }
  void plan_implicit_setup(std::vector<Pass>& out) {
    const int M1 = c->opt.order - 1;
    out.push_back(plan_col_a());   // V1 = F{V^(1)}, grad phi~ (mixed)
    RowB r = row_begin();
    for (char d : dims()) {
      c2r(r, 0, {std::string("dphi") + d});
      for (int b = 0; b <= M1; ++b)
        prod(r, 0, b ? 1 : 0, 0, b ? 2 : 0, 1.0, S("IP%d", b) + d);   // eta^b grad phi~
    }
    out.push_back(row_end(r, true, false, false));
    const std::vector<bool> has = plan_inner(out, M1 + 1, "IGS", inner_eta_inputs(false, "IP%d"));
    plan_implicit_outer(out, has, "IGS", "IGU");
    plan_implicit_sum(out, has, "IGS", "IGU", {{st_phi, {term(0, 1.0, 1, 1, 0, 0)}}}, "IG", {});
  }
  // Variable bottom (Appendices A and B together): the unknowns V and the
  // bottom potential varphi~, iterated as V and grad varphi~ (mixed).  With
  // m the order of a term (j = m + 1):
  //   V^(j) += C_h k 2 (-1)^a/(a! b!) F{eta^a F^{-1}{sqrt(e_h) k^{j-3} ik.F{delta^b grad varphi~}}}, b odd;
  //   varphi~^(j) = D_h ( 2/(a! c!) F{delta^c F^{-1}{sqrt(e_h) k^{j-2} F{eta^a V}}}          (a even)
  //                     + 2/(a! c!) F{delta^c F^{-1}{sqrt(e_h) k^{j-3} ik.F{eta^a grad phi~}}} (a odd)
  //                     + s/(c! b!) F{delta^c F^{-1}{X k^{j-3} ik.F{delta^b grad varphi~}}} (j >= 2) ),
  // s X = -C_h^{-1} (b odd), +D_h^{-1} (b even), and -e_h for every term of
  // varphi~^(5) (the printed form; the same operator).
  bool bottom_self_term(int acc, int cpow, int b, int gx, int gy, ColTerm* t) const {
    const int j = cpow + b + 1;
    if (j < 2 || j > c->opt.order - 1) return false;
    const double f = fact(cpow) * fact(b);
    if (j == 5) *t = term(acc, -1.0 / f, j - 3, 10, gx, gy, 1);
    else if (b % 2) *t = term(acc, -1.0 / f, j - 3, 8, gx, gy, 1);
    else *t = term(acc, 1.0 / f, j - 3, 9, gx, gy, 1);
    return true;
  }
  // F{eta^a F^{-1}{S_a}} (a >= 1) and F{delta^c F^{-1}{T_c}} (c >= 1) by one row pass
  void plan_implicit_outer2(std::vector<Pass>& out, const std::vector<bool>& has_s, const std::string& ps,
                            const std::string& pu, const std::vector<bool>& has_t, const std::string& pt,
                            const std::string& pw) {
    RowB r = row_begin();
    bool any = false;
    for (size_t a = 1; a < has_s.size(); ++a)
      if (has_s[a]) {
        c2r(r, 0, {ps + std::to_string(a)});
        prod(r, 0, (int)a, 0, 0, 1.0, pu + std::to_string(a));
        any = true;
      }
    for (size_t cc = 1; cc < has_t.size(); ++cc)
      if (has_t[cc]) {
        c2r(r, 0, {pt + std::to_string(cc)});
        prod(r, 0, 0, (int)cc, 0, 1.0, pw + std::to_string(cc));
        any = true;
      }
    if (any) out.push_back(row_end(r, true, true, false));
  }
  // D_h (nx T_0 + sum_{c>=1} F{delta^c t_c}) (+ extra inputs) as its gradient
  // (ik, masked) in dst_x, dst_y, or as the spectrum itself in dst_x when
  // gradient is false
  void plan_bottom_sum(std::vector<Pass>& out, const std::vector<bool>& has, const std::string& pt,
                       const std::string& pw, std::vector<ColIn> ins, const std::string& dst_x,
                       const std::string& dst_y, bool gradient) {
    if (!has.empty() && has[0]) ins.push_back({pt + "0", {term(0, (double)g.nx, 0, 13, 0, 0)}});
    for (size_t cc = 1; cc < has.size(); ++cc)
      if (has[cc]) ins.push_back({pw + std::to_string(cc), {term(0, 1.0, 0, 13, 0, 0)}});
    std::vector<std::pair<std::string, ColTerm>> outs;
    if (!gradient) {
      outs.push_back({dst_x, term(0, 1.0, 0, 0, 0, 0, 1)});
    } else {
      outs.push_back({dst_x, term(0, 1.0, 0, 0, 1, 0, 1)});
      if (g.two_d) outs.push_back({dst_y, term(0, 1.0, 0, 0, 0, 1, 1)});
    }
    out.push_back(col(ins, outs, 1));
  }
  void plan_implicit_setup_var(std::vector<Pass>& out) {
    plan_implicit_setup(out);   // V1, grad varphi~_1 (db1), eta^b grad phi~ (IP), G_V (IG)
    const int M1 = c->opt.order - 1;
    std::vector<std::pair<std::string, TermFn>> ins;
    for (int a = 1; a <= M1; a += 2)
      for (char d : dims())
        ins.push_back({S("IP%d", a) + d, [this, a, d, M1](int cc, int acc, ColTerm* t) {
                         const int j = a + cc + 1;
                         if (j > M1) return false;
                         *t = term(acc, 2.0 / (fact(a) * fact(cc)), j - 3, 12, d == 'x', d == 'y', 1);
                         return true;
                       }});
    const std::vector<bool> has = plan_inner(out, M1, "IGT", ins);
    plan_implicit_outer2(out, {}, "", "", has, "IGT", "IGW");
    plan_bottom_sum(out, has, "IGT", "IGW", {}, "IGB", "", false);
  }
  void plan_implicit_iter_var(std::vector<Pass>& out, const std::string& srcV, const std::string& srcBx,
                              const std::string& srcBy, const std::string& dstV, const std::string& dstBx,
                              const std::string& dstBy) {
    const int M1 = c->opt.order - 1;
    RowB r = row_begin();
    c2r(r, 0, {srcV});
    for (int b = 0; b <= M1; ++b) prod(r, 0, b ? 1 : 0, 0, b ? 2 : 0, 1.0, S("IQ%d", b));   // eta^b V
    for (char d : dims()) {
      c2r(r, 0, {d == 'x' ? srcBx : srcBy});
      for (int b = 0; b <= M1; ++b) prod(r, 0, 0, b ? 1 : 0, b ? 2 : 0, 1.0, S("IR%d", b) + d);   // delta^b grad varphi~
    }
    out.push_back(row_end(r, true, true, false));
    // V equation: S_a from eta^b V and (odd b) delta^b grad varphi~
    std::vector<std::pair<std::string, TermFn>> vin = inner_eta_inputs(true, "IQ%d");
    for (int b = 1; b <= M1; b += 2)
      for (char d : dims())
        vin.push_back({S("IR%d", b) + d, [this, b, d, M1](int a, int acc, ColTerm* t) {
                         if (a + b > M1) return false;
                         *t = term(acc, ((a % 2) ? -2.0 : 2.0) / (fact(a) * fact(b)), a + b - 2, 12, d == 'x',
                                   d == 'y', 1);
                         return true;
                       }});
    const std::vector<bool> has_s = plan_inner(out, M1 + 1, "IS", vin);
    // varphi~ equation: T_c from (even a) eta^a V and delta^b grad varphi~
    std::vector<std::pair<std::string, TermFn>> bin;
    for (int a = 0; a <= M1; a += 2)
      bin.push_back({S("IQ%d", a), [this, a, M1](int cc, int acc, ColTerm* t) {
                       const int j = a + cc + 1;
                       if (j > M1) return false;
                       *t = term(acc, 2.0 / (fact(a) * fact(cc)), j - 2, 12, 0, 0, 1);
                       return true;
                     }});
    for (int b = 0; b <= M1; ++b)
      for (char d : dims())
        bin.push_back({S("IR%d", b) + d, [this, b, d](int cc, int acc, ColTerm* t) {
                         return bottom_self_term(acc, cc, b, d == 'x', d == 'y', t);
                       }});
    const std::vector<bool> has_t = plan_inner(out, M1, "IT", bin);
    plan_implicit_outer2(out, has_s, "IS", "IU", has_t, "IT", "IW");
    plan_implicit_sum(out, has_s, "IS", "IU", {}, dstV, {"IG"});
    // G_B enters as a column output (spectrum / nx): scaled by nx
    plan_bottom_sum(out, has_t, "IT", "IW", {{"IGB", {term(0, (double)g.nx, 0, 0, 0, 0)}}}, dstBx, dstBy, true);
  }
  void plan_implicit_iter(std::vector<Pass>& out, const std::string& src, const std::string& dst) {
    const int M1 = c->opt.order - 1;
    RowB r = row_begin();
    c2r(r, 0, {src});
    for (int b = 0; b <= M1; ++b) prod(r, 0, b ? 1 : 0, 0, b ? 2 : 0, 1.0, S("IQ%d", b));   // eta^b V
    out.push_back(row_end(r, true, false, false));
    const std::vector<bool> has = plan_inner(out, M1 + 1, "IS", inner_eta_inputs(true, "IQ%d"));
    plan_implicit_outer(out, has, "IS", "IU");
    plan_implicit_sum(out, has, "IS", "IU", {}, dst, {"IG"});
  }
};


// ---------------------------------------------------------------------------
// Adaptive-order convergence test (phases of ConvParams)
// ---------------------------------------------------------------------------
__global__ void k_conv_reset(ConvParams q, int order) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= q.n) return;
  q.conv[m] = 1;
  q.orders[m] = order;
  q.notconv[m] = 0;
}

// Parseval weights on the mixed layout: kx = 0 once, kx > 0 twice (the
// conjugate modes); the common factor ny cancels in the ratio.
template <typename T>
__global__ void k_conv_norms(ConvParams q) {
  using V = cx<T>;
  __shared__ double sm[2][256];
  const int m = blockIdx.y;
  double inc = 0.0, tot = 0.0;
  if (q.conv[m]) {
    const long long ne = (long long)q.W * q.ny;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (long long)gridDim.x * blockDim.x) {
      const double w = (e / q.ny) == 0 ? 1.0 : 2.0;
      double sr = 0.0, si = 0.0, lr = 0.0, li = 0.0;
      for (int l = 0; l < q.nlev; ++l) {
        const V v = reinterpret_cast<const V*>(q.V[l])[m * q.stride + e];
        sr += double(v.x);
        si += double(v.y);
        if (l == q.nlev - 1) { lr = double(v.x); li = double(v.y); }
      }
      if (q.last) {   // V_M = Vsum - (V_1 + .. + V_{M-1})
        const V t = reinterpret_cast<const V*>(q.vsum)[m * q.stride + e];
        lr = double(t.x) - sr;
        li = double(t.y) - si;
        sr = double(t.x);
        si = double(t.y);
      }
      inc += w * (lr * lr + li * li);
      tot += w * (sr * sr + si * si);
    }
  }
  sm[0][threadIdx.x] = inc;
  sm[1][threadIdx.x] = tot;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + st];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    q.red[(m * kConvBlocks + blockIdx.x) * 2] = sm[0][0];
    q.red[(m * kConvBlocks + blockIdx.x) * 2 + 1] = sm[1][0];
  }
}

__device__ __forceinline__ bool conv_meets(const ConvParams& q, int m) {
  double inc = 0.0, tot = 0.0;
  for (int b = 0; b < kConvBlocks; ++b) {   // fixed order
    inc += q.red[(m * kConvBlocks + b) * 2];
    tot += q.red[(m * kConvBlocks + b) * 2 + 1];
  }
  return inc <= q.tol2 * tot;
}

template <typename T>
__global__ void k_conv_write(ConvParams q) {
  using V = cx<T>;
  __shared__ int go;
  const int m = blockIdx.y;
  if (threadIdx.x == 0) go = q.conv[m] && conv_meets(q, m);
  __syncthreads();
  if (!go) return;
  const long long ne = (long long)q.W * q.ny;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    V s = mk<V>(T(0), T(0));
    for (int l = 0; l < q.nlev; ++l) s = cadd(s, reinterpret_cast<const V*>(q.V[l])[m * q.stride + e]);
    reinterpret_cast<V*>(q.vsum)[m * q.stride + e] = s;
  }
}

__global__ void k_conv_update(ConvParams q) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= q.n || !q.conv[m]) return;
  if (conv_meets(q, m)) {
    q.conv[m] = 0;
    q.orders[m] = q.level;
  } else if (q.last) {
    q.notconv[m] = 1;
  }
}

// Wavemaker pressure at a stage time (FP64 sums and sines: omega t reaches
// thousands of radians), rounded once to the working precision.
template <typename T>
__global__ void k_wavemaker(WmkParams q) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= q.nx) return;
  const double t = *q.t + q.offset;
  double acc = 0.0;
  for (int j = 0; j < q.J; ++j) acc += q.prof[(size_t)j * q.nx + x] * sin(q.omega[j] * t + q.phase[j]);
  reinterpret_cast<T*>(q.out)[x] = T(acc);
}

__global__ void k_advance_time(double* t, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t += dt;
}

// Step norms of the adaptive scheme: block partials in a fixed order, then
// one thread per member sums the partials in block order.
template <typename T>
__global__ void k_norm45_partials(NormParams q) {
  using V = cx<T>;
  __shared__ double sm[4][256];
  const int m = blockIdx.y;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long ne = (long long)q.W * q.ny;
  const V* src[4] = {reinterpret_cast<const V*>(q.ee), reinterpret_cast<const V*>(q.ep),
                     reinterpret_cast<const V*>(q.ue), reinterpret_cast<const V*>(q.up)};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const double w = (e / q.ny) == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const V v = src[f][m * q.stride + e];
      acc[f] += w * ((double)v.x * v.x + (double)v.y * v.y);
    }
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] = acc[f];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
#pragma unroll
      for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] += sm[f][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 4) q.part[((size_t)m * kConvBlocks + blockIdx.x) * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

// Increment norms of the implicit iteration, one block per member: the
// Parseval sums of |a - b|^2 and |a|^2 over the member's mixed field (kx = 0
// once, kx > 0 twice), reduced in a fixed order.
constexpr int kImplicitMaxIter = 64;
template <typename T>
__global__ void k_implicit_norms(const void* a, const void* b, long long stride, int W, int ny, double* out) {
  using V = cx<T>;
  __shared__ double sm[2][256];
  const int m = blockIdx.x;
  const V* pa = reinterpret_cast<const V*>(a) + m * stride;
  const V* pb = reinterpret_cast<const V*>(b) + m * stride;
  double d2 = 0.0, a2 = 0.0;
  const long long ne = (long long)W * ny;
  for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
    const double w = (e / ny) == 0 ? 1.0 : 2.0;
    const V u = pa[e], v = pb[e];
    const double dr = double(u.x) - double(v.x), di = double(u.y) - double(v.y);
    d2 += w * (dr * dr + di * di);
    a2 += w * (double(u.x) * double(u.x) + double(u.y) * double(u.y));
  }
  sm[0][threadIdx.x] = d2;
  sm[1][threadIdx.x] = a2;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + st];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * m] = sm[0][0];
    out[2 * m + 1] = sm[1][0];
  }
}

// Crest of one member: the largest sample of eta (the first in row-major
// order among equal samples), found by one block in a fixed order, and its
// position refined along each axis by the parabola through the sample and
// its periodic neighbours; out = (x, y, height), NaN when no sample compares
// (a non-finite state).
__device__ __forceinline__ double crest_shift(double fm, double f0, double fp) {
  const double den = fm - 2.0 * f0 + fp;
  return den != 0.0 ? 0.5 * (fm - fp) / den : 0.0;
}
__global__ void k_crest(const double* __restrict__ f, int nx, int ny, double dx, double dy, double* out) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  const int t = threadIdx.x;
  const long long np = (long long)nx * ny;
  double best = -INFINITY;
  long long bi = np;
  for (long long e = t; e < np; e += blockDim.x) {
    const double v = f[e];
    if (v > best) {   // a thread visits increasing e: the first maximum stays
      best = v;
      bi = e;
    }
  }
  sv[t] = best;
  si[t] = bi;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (t < st) {
      const double v2 = sv[t + st];
      const long long i2 = si[t + st];
      if (v2 > sv[t] || (v2 == sv[t] && i2 < si[t])) {
        sv[t] = v2;
        si[t] = i2;
      }
    }
    __syncthreads();
  }
  if (t != 0) return;
  const long long e = si[0];
  if (e >= np) {
    out[0] = out[1] = out[2] = NAN;
    return;
  }
  const int j = (int)(e / nx), i = (int)(e % nx);
  const double f0 = f[e];
  out[0] = (i + crest_shift(f[(long long)j * nx + (i + nx - 1) % nx], f0, f[(long long)j * nx + (i + 1) % nx])) * dx;
  out[1] = ny > 1 ? (j + crest_shift(f[(long long)((j + ny - 1) % ny) * nx + i], f0,
                                     f[(long long)((j + 1) % ny) * nx + i])) * dy
                  : 0.0;
  out[2] = f0;
}

__global__ void k_norm45_finish(NormParams q) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= q.n) return;
  for (int f = 0; f < 4; ++f) {
    double s = 0.0;
    for (int b = 0; b < kConvBlocks; ++b) s += q.part[((size_t)m * kConvBlocks + b) * 4 + f];
    q.out[m * 4 + f] = s;
  }
}

// ---------------------------------------------------------------------------
// Execution
// ---------------------------------------------------------------------------
int launch_pass(sbi_ctx* c, const Pass& p, cudaStream_t st) {
  if (p.kind == PK_NORM) {
    const NormParams& q = p.norm;
    if (c->fp64) k_norm45_partials<double><<<dim3(kConvBlocks, q.n), 256, 0, st>>>(q);
    else k_norm45_partials<float><<<dim3(kConvBlocks, q.n), 256, 0, st>>>(q);
    k_norm45_finish<<<(q.n + 127) / 128, 128, 0, st>>>(q);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SBI_OK : cuda_fail(c, e, "kernel launch");
  }
  if (p.kind == PK_WMK) {
    const WmkParams& q = p.wmk;
    if (c->fp64) k_wavemaker<double><<<(q.nx + 255) / 256, 256, 0, st>>>(q);
    else k_wavemaker<float><<<(q.nx + 255) / 256, 256, 0, st>>>(q);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SBI_OK : cuda_fail(c, e, "kernel launch");
  }
  cudaError_t e = cudaSuccess;
  if (p.kind == PK_CONV) {
    const ConvParams& q = p.conv;
    const dim3 grid(kConvBlocks, q.n);
    switch (q.phase) {
      case 0: k_conv_reset<<<(q.n + 255) / 256, 256, 0, st>>>(q, c->opt.order); break;
      case 1:
        if (c->fp64) k_conv_norms<double><<<grid, 256, 0, st>>>(q);
        else k_conv_norms<float><<<grid, 256, 0, st>>>(q);
        break;
      case 2:
        if (c->fp64) k_conv_write<double><<<grid, 256, 0, st>>>(q);
        else k_conv_write<float><<<grid, 256, 0, st>>>(q);
        break;
      default: k_conv_update<<<(q.n + 255) / 256, 256, 0, st>>>(q); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return SBI_OK;
  }
  if (p.kind == PK_ROW) e = c->fp64 ? launch_row<double>(p.nsize, p.row, st) : launch_row<float>(p.nsize, p.row, st);
  else if (p.kind == PK_COL) e = c->fp64 ? launch_col<double>(p.nsize, p.col, st) : launch_col<float>(p.nsize, p.col, st);
  else e = c->fp64 ? launch_rk<double>(p.nsize, p.rk, st) : launch_rk<float>(p.nsize, p.rk, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return SBI_OK;
}

int run_passes(sbi_ctx* c, const std::vector<Pass>& ps, cudaStream_t st) {
  for (auto& p : ps) {
    int rc = launch_pass(c, p, st);
    if (rc) return rc;
  }
  return SBI_OK;
}

// ---------------------------------------------------------------------------
// Autotuner.  A row pass may run with any power-of-two number of rows per
// block up to the planner's choice, a column pass with any number of columns
// per block up to the size's default, as long as a block is made of whole
// warps.  Neither changes the arithmetic of a row or a column, so the results
// are the same bits for every choice; only the split into blocks (occupancy,
// tail of the last wave) changes.  Each distinct pass shape is timed once on
// the real buffers (one warm-up and three timed launches per candidate) and
// the fastest is kept; the planner's default stays unless another candidate
// is at least 3 % faster.  Passes whose outputs alias their inputs (not
// idempotent, e.g. an in-place filter) are never re-run and keep the default.
// ---------------------------------------------------------------------------
bool pass_idempotent(const Pass& p) {
  std::vector<const void*> in, out;
  if (p.kind == PK_ROW) {
    const RowParams& r = p.row;
    for (int o = 0; o < r.nops; ++o) {
      const RowOp& op = r.ops[o];
      if (op.kind == ROP_C2R) {
        for (int q = 0; q < op.b; ++q) in.push_back(r.buf[op.a + q].ptr);
        if (op.dst != kNone) out.push_back(r.buf[op.dst].ptr);
      } else {
        out.push_back(r.buf[op.dst].ptr);
      }
    }
    in.push_back(r.eta.ptr);
    in.push_back(r.delta.ptr);
    in.push_back(r.wgt.ptr);
  } else if (p.kind == PK_COL) {
    const ColParams& q = p.col;
    for (int i = 0; i < q.nin; ++i) in.push_back(q.buf[i].ptr);
    for (int i = 0; i < q.npass; ++i) in.push_back(q.pass[i].ptr);
    for (int o = 0; o < q.nouts; ++o) out.push_back(q.buf[q.nin + o].ptr);
    if (q.norm_out) return false;
  } else {
    return false;
  }
  for (const void* a : out)
    for (const void* b : in)
      if (a && a == b) return false;
  return true;
}

std::string pass_signature(const Pass& p) {
  char b[160];
  if (p.kind == PK_ROW) {
    std::string ops;
    for (int o = 0; o < p.row.nops; ++o) ops += "CPNWV"[p.row.ops[o].kind < 5 ? p.row.ops[o].kind : 0];
    snprintf(b, sizeof(b), "row nx=%d rows=%d slots=%d ops=%d ", p.nsize, p.row.rows_total - p.row.row_begin,
             p.row.nslots, p.row.nops);
    return b + ops;
  }
  snprintf(b, sizeof(b), "col ny=%d cols=%d in=%d terms=%d out=%d acc=%d pass=%d", p.nsize,
           p.col.cols_total - p.col.col_begin, p.col.nin, p.col.nterms, p.col.nouts, p.col.nacc, p.col.npass);
  return b;
}

constexpr int kStagedTag = 1 << 16;

int tune_pass(sbi_ctx* c, Pass& p, cudaStream_t st) {
  if (!c->opt.autotune || (p.kind != PK_ROW && p.kind != PK_COL)) return SBI_OK;
  // a column choice packs the columns per block and the staged form (bulk
  // copies of the inputs into shared memory) as cpb + kStagedTag * staged
  auto apply = [&](Pass& q, int v) {
    if (q.kind == PK_ROW) {
      q.row.rpc = v;
    } else {
      q.col.cpb = v % kStagedTag;
      q.col.staged = v / kStagedTag;
    }
  };
  const std::string key = pass_signature(p);
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) {
    apply(p, it->second.choice);
    return SBI_OK;
  }
  std::vector<int> cand;
  int deflt = 0;
  if (p.kind == PK_ROW) {
    const int tpr = c->fp64 ? row_tpr<double>(p.nsize) : row_tpr<float>(p.nsize);
    deflt = p.row.rpc;
    for (int r = deflt; r >= 1 && cand.size() < 4; r /= 2)
      if (tpr > 0 && (r * tpr) % 32 == 0) cand.push_back(r);
  } else {
    int tpc = 0;
    const int cpb = c->fp64 ? col_geometry<double>(p.nsize, &tpc) : col_geometry<float>(p.nsize, &tpc);
    const int base = p.col.cpb > 0 ? p.col.cpb : cpb;
    deflt = base + kStagedTag * p.col.staged;
    // the staged form is a candidate where the option leaves the choice open
    const bool stg = c->opt.col_staging == 0 &&
                     (c->fp64 ? col_stageable<double>(p.nsize) : col_stageable<float>(p.nsize));
    for (int staged = p.col.staged; staged <= (stg ? 1 : p.col.staged); ++staged) {
      int k = 0;
      for (int v = base; v >= 1 && k < 3; v /= 2)
        if (tpc > 0 && (v * tpc) % 32 == 0) {
          cand.push_back(v + kStagedTag * staged);
          ++k;
        }
    }
  }
  int best = deflt;
  double best_ms = -1.0, deflt_ms = -1.0;
  if (cand.size() > 1 && pass_idempotent(p)) {
    if (!c->tune_ev[0]) {
      CK(cudaEventCreate(&c->tune_ev[0]), "event");
      CK(cudaEventCreate(&c->tune_ev[1]), "event");
    }
    for (int v : cand) {
      Pass q = p;
      apply(q, v);
      int rc = launch_pass(c, q, st);  // warm-up
      if (rc) return rc;
      CK(cudaEventRecord(c->tune_ev[0], st), "event");
      for (int k = 0; k < 3; ++k) {
        rc = launch_pass(c, q, st);
        if (rc) return rc;
      }
      CK(cudaEventRecord(c->tune_ev[1], st), "event");
      CK(cudaEventSynchronize(c->tune_ev[1]), "tuning sync");
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]), "event time");
      const double t = ms / 3.0;
      if (v == deflt) deflt_ms = t;
      if (best_ms < 0.0 || t < best_ms) {
        best_ms = t;
        best = v;
      }
    }
    if (best != deflt && !(best_ms < 0.97 * deflt_ms)) {
      best = deflt;
      best_ms = deflt_ms;
    }
  }
  c->tuned[key] = sbi_ctx::Tuned{best, deflt, best_ms};
  c->tune_order.push_back(key);
  apply(p, best);
  return SBI_OK;
}

// Passes of one step for each member group (groups are independent).
std::vector<std::vector<Pass>> plan_step_groups(sbi_ctx* c, double dt, bool* oom, int kind = SK_STEP) {
  std::vector<std::vector<Pass>> out;
  for (auto& g : c->groups) {
    std::vector<Pass> all;
    Planner pl{c, g};
    if (kind == SK_RK45_A) {
      // six stages: the diagnostic and right-hand side of stage i give k_i;
      // the offsets of stage i + 1 follow; then the order-5 offsets, the
      // error offsets and the step norms
      for (int s = 1; s <= 6; ++s) {
        pl.if_stage = s;
        pl.st_eta = s == 1 ? "eta_m" : "eta_s";
        pl.st_phi = s == 1 ? "phi_m" : "phi_s";
        pl.st_eta_w = s == 1 ? nullptr : pl.stage_eta_w();
        pl.plan_diag(all);
        pl.plan_rhs(all, 0.0);
        pl.if_stage = 0;
        pl.st_eta = "eta_m";
        pl.st_phi = "phi_m";
        pl.st_eta_w = nullptr;
        if (s < 6) {
          all.push_back(pl.plan_ck_combine(s + 1));
          all.push_back(pl.plan_rk(RK_OFFSET, s, 0.0, 1, "De", "Dp", "eta_s", "phi_s", pl.stage_eta_w()));
        }
      }
      all.push_back(pl.plan_ck_combine(7));
      all.push_back(pl.plan_ck_combine(8));
      all.push_back(pl.plan_norm45());
      if (pl.oom) *oom = true;
      out.push_back(std::move(all));
      continue;
    }
    if (kind == SK_RK45_B) {
      // accept the step: the order-5 offsets into the state
      // the accepted state's working copies come from this pass's tail; the
      // filter's projection then needs no entry pass of its own
      all.push_back(pl.plan_rk(RK_CORRECT, 4, 0.0, 1, "De", "Dp"));
      if (c->filter_on()) pl.plan_project(all, true, false);
      if (pl.oom) *oom = true;
      out.push_back(std::move(all));
      continue;
    }
    for (int s = 1; s <= 4; ++s) {
      const double t_off = (s == 1 ? 0.0 : (s == 4 ? 1.0 : 0.5)) * dt;  // stage times
      // every stage's tail writes the working copies of its state; after the
      // last stage they are those of the new state, which the filter's
      // projection reads (so it needs no entry pass)
      const int tail = 1;
      if (c->opt.integrator == SBI_LAWSON_RK4) {
        // integrating factor: stage 1 is u_n (eta_m, phi_m), the later stages'
        // working copies live in (eta_s, phi_s)
        pl.if_stage = s;
        pl.st_eta = s == 1 ? "eta_m" : "eta_s";
        pl.st_phi = s == 1 ? "phi_m" : "phi_s";
        pl.plan_diag(all);
        pl.plan_rhs(all, t_off);
        all.push_back(pl.plan_if_combine(s, dt));
        if (s < 4) all.push_back(pl.plan_rk(RK_OFFSET, s, dt, 1, "De", "Dp", "eta_s", "phi_s"));
        else all.push_back(pl.plan_rk(RK_CORRECT, s, dt, tail, "De", "Dp"));
        pl.if_stage = 0;
        pl.st_eta = "eta_m";
        pl.st_phi = "phi_m";
      } else {
        pl.plan_diag(all);
        pl.plan_rhs(all, t_off);
        all.push_back(pl.plan_rk(RK_STAGE, s, dt, tail));
      }
    }
    if (c->filter_on()) pl.plan_project(all, true, false);
    if (pl.oom) *oom = true;
    out.push_back(std::move(all));
  }
  return out;
}

// ---------------------------------------------------------------------------
// Step schedule.  The members of a group are independent problems, so the
// passes of a step can run over any partition of the batch into units (member
// ranges of one group), as concurrent graph branches or one unit after
// another: the arithmetic of every member is the same in every case, and so
// are the results, bit for bit.  What changes is how the launches fill the
// GPU (launch sizes, the tails of their last waves, overlap between branches).
// The candidates are the serial order, one branch per group, and splits of the
// groups into nearly equal member ranges of at most total/B points for
// B = 2, 3, 4, 6; B = 3 is the default.  On the first step of the classical
// RK4 or Lawson scheme, with autotuning on, every candidate's step graph is
// captured and timed on the real buffers (one warm-up and three timed replays,
// the state saved before and restored after), and the fastest is kept; the
// default stays unless another candidate is at least 3 % faster.
// ---------------------------------------------------------------------------
bool pass_sliceable(const Pass& p) { return p.kind == PK_ROW || p.kind == PK_COL || p.kind == PK_RK; }

// a group's pass restricted to its members [m0, m1)
Pass slice_pass(const Pass& p, const Group& g, int m0, int m1) {
  Pass q = p;
  if (m0 == 0 && m1 == g.n) return q;
  if (p.kind == PK_ROW) {
    q.row.row_begin = m0 * g.ny;
    q.row.rows_total = m1 * g.ny;
  } else if (p.kind == PK_COL) {
    q.col.col_begin = m0 * g.W;
    q.col.cols_total = m1 * g.W;
  } else {
    q.rk.row_begin = m0 * g.ny;
    q.rk.rows_total = m1 * g.ny;
  }
  const double f = (double)(m1 - m0) / (double)g.n;
  q.bytes *= f;
  q.xforms *= f;
  return q;
}

struct Sched {
  std::vector<Unit> units;
  bool serial;
  std::string name;
};

// Units with at most cap points each (cap 0: one unit per group); only
// groups whose passes can all be sliced are split.
std::vector<Unit> units_for_cap(const sbi_ctx* c, size_t cap, const std::vector<bool>& sliceable) {
  std::vector<size_t> pts;
  std::vector<int> n;
  for (const Group& g : c->groups) {
    pts.push_back(g.phys_elems() * (size_t)g.n);
    n.push_back(g.n);
  }
  return sbi::units_for_cap(pts, n, cap, sliceable);
}

// which groups' step passes can all be restricted to member ranges
std::vector<bool> groups_sliceable(sbi_ctx* c, bool* oom) {
  std::vector<bool> ok(c->groups.size(), true);
  std::vector<int> kinds = {SK_STEP};
  if (c->opt.integrator == SBI_IF_RK45) kinds = {SK_RK45_A, SK_RK45_B};
  for (int kind : kinds) {
    const std::vector<std::vector<Pass>> gps = plan_step_groups(c, 1.0, oom, kind);
    for (size_t gi = 0; gi < gps.size(); ++gi)
      for (const Pass& p : gps[gi])
        if (!pass_sliceable(p)) ok[gi] = false;
  }
  return ok;
}

// the candidate schedules, the default first
std::vector<Sched> sched_candidates(sbi_ctx* c, bool* oom) {
  const std::vector<bool> sl = groups_sliceable(c, oom);
  size_t total = 0, biggest = 0;
  for (const auto& g : c->groups) {
    total += g.phys_elems() * (size_t)g.n;
    biggest = std::max(biggest, g.phys_elems());
  }
  std::vector<Sched> out;
  auto add = [&](std::vector<Unit> u, bool serial, const std::string& name) {
    if (u.size() < 2) serial = false;   // one unit: the same graph either way
    for (const auto& s2 : out)
      if (s2.units == u && s2.serial == serial) return;
    out.push_back(Sched{std::move(u), serial, name});
  };
  auto cap_of = [&](size_t B) { return std::max(biggest, (total + B - 1) / B); };
  add(units_for_cap(c, cap_of(3), sl), false, "split total/3");
  add(units_for_cap(c, 0, sl), true, "serial groups");
  add(units_for_cap(c, 0, sl), false, "one branch per group");
  for (size_t B : {2, 4, 6}) add(units_for_cap(c, cap_of(B), sl), false, "split total/" + std::to_string(B));
  return out;
}

// the schedule opt.schedule names (-1: serial groups; B > 0: split total/B)
Sched forced_sched(sbi_ctx* c, bool* oom) {
  const std::vector<bool> sl = groups_sliceable(c, oom);
  size_t total = 0, biggest = 0;
  for (const auto& g : c->groups) {
    total += g.phys_elems() * (size_t)g.n;
    biggest = std::max(biggest, g.phys_elems());
  }
  const int B = c->opt.schedule;
  Sched s{B < 0 ? units_for_cap(c, 0, sl)
                : units_for_cap(c, std::max(biggest, (total + (size_t)B - 1) / (size_t)B), sl),
          B < 0, B < 0 ? "serial groups" : "split total/" + std::to_string(B)};
  if (s.units.size() < 2) s.serial = false;
  return s;
}

// The passes of one step per unit of the current schedule (before the
// schedule is chosen: the named one, else the default).
std::vector<std::vector<Pass>> plan_step_units(sbi_ctx* c, double dt, bool* oom, int kind = SK_STEP) {
  if (c->units.empty()) {
    const Sched s = c->opt.schedule != 0 ? forced_sched(c, oom) : sched_candidates(c, oom)[0];
    c->units = s.units;
    c->serial = s.serial;
  }
  const std::vector<std::vector<Pass>> gps = plan_step_groups(c, dt, oom, kind);
  std::vector<std::vector<Pass>> out;
  for (const Unit& u : c->units) {
    const Group& g = c->groups[u.group];
    std::vector<Pass> v;
    for (const Pass& p : gps[u.group]) v.push_back(slice_pass(p, g, u.m0, u.m1));
    out.push_back(std::move(v));
  }
  return out;
}

std::vector<Pass> plan_step(sbi_ctx* c, double dt, bool* oom) {
  std::vector<Pass> all;
  if (c->opt.integrator == SBI_IF_RK45) {
    for (int kind : {SK_RK45_A, SK_RK45_B})
      for (auto& v : plan_step_units(c, dt, oom, kind)) all.insert(all.end(), v.begin(), v.end());
    return all;
  }
  for (auto& v : plan_step_units(c, dt, oom)) all.insert(all.end(), v.begin(), v.end());
  return all;
}

// Write the values of the h-dependent tables for the step h (stream-ordered
// before the graph that reads them).
int update_dyn_tables(sbi_ctx* c, double h, cudaStream_t st) {
  if (h == c->dyn_h) return SBI_OK;
  for (auto& g : c->groups)
    for (const auto& d : g.dyn) {
      TableSpec s = d.spec;
      s.tau = d.r * h;
      s.c = d.spec.c * (d.p ? h : 1.0);
      const cudaError_t e = c->fp64 ? launch_coef_table<double>(d.ptr, s, st)
                                    : launch_coef_table<float>(d.ptr, s, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "table kernel");
    }
  c->dyn_h = h;
  return SBI_OK;
}

int family_of(const Pass& p) {
  switch (p.kind) {
    case PK_COL: return FAM_COL;
    case PK_ROW: return FAM_ROW;
    case PK_RK: return FAM_RK;
    case PK_WMK: return FAM_WMK;
    default: return FAM_CONV;   // adaptive-order tests and step norms
  }
}

void free_graphs(sbi_ctx* c) {
  for (auto& ge : c->graphs) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    if (ge.graph) cudaGraphDestroy(ge.graph);
    for (auto e : ge.ev) cudaEventDestroy(e);
  }
  c->graphs.clear();
}

// Capture the step graph of the current schedule (only == nullptr: every
// unit), or of one member range alone (the streamed step).
int build_step_graph(sbi_ctx* c, double dt, int kind, const Unit* only, GraphEntry& ge) {
  bool oom = false;
  std::vector<std::vector<Pass>> gps;
  if (only) {
    const std::vector<std::vector<Pass>> all = plan_step_groups(c, dt, &oom, kind);
    std::vector<Pass> one;
    for (const Pass& p : all.at((size_t)only->group))
      one.push_back(slice_pass(p, c->groups[only->group], only->m0, only->m1));
    gps.push_back(std::move(one));
  } else {
    gps = plan_step_units(c, dt, &oom, kind);
  }
  if (oom) return fail(c, SBI_ENOMEM, "device allocation failed while planning the step");
  CK(cudaStreamSynchronize(c->cap), "sync before capture");
  CK(cudaStreamSynchronize(c->stream), "sync before capture");
  // block shapes are tuned (or taken from earlier tuning) before capture
  for (auto& v : gps)
    for (auto& p : v) {
      const int rc = tune_pass(c, p, c->cap);
      if (rc) return rc;
    }
  size_t npasses = 0;
  for (auto& v : gps) npasses += v.size();
  ge.dt = dt;
  ge.prof = c->prof;
  ge.kind = kind;
  ge.group = only ? only->group : -1;
  ge.m0 = only ? only->m0 : 0;
  ge.m1 = only ? only->m1 : 0;
  if (c->prof) {   // the profiled graph owns one event pair per pass
    for (size_t gi = 0; gi < gps.size(); ++gi)
      for (size_t i = 0; i < gps[gi].size(); ++i) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a), "event");
        CK(cudaEventCreate(&b), "event");
        ge.ev.push_back(a);
        ge.ev.push_back(b);
        ge.ev_family.push_back(family_of(gps[gi][i]));
      }
  }
  // one branch per unit: fork from the capture stream, join back
  while (c->gstreams.size() < gps.size()) {
    cudaStream_t s2;
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "stream");
    c->gstreams.push_back(s2);
  }
  while (c->gevents.size() < gps.size() + 1) {
    cudaEvent_t e2;
    CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "event");
    c->gevents.push_back(e2);
  }
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = SBI_OK;
  // the units run as concurrent branches unless the schedule is serial; a
  // profiled replay runs them one after the other, so that each launch's
  // event pair times that launch alone
  const bool branch = gps.size() > 1 && !c->prof && !c->serial;
  if (branch) cudaEventRecord(c->gevents[0], c->cap);
  size_t evi = 0;
  for (size_t gi = 0; gi < gps.size() && rc == SBI_OK; ++gi) {
    cudaStream_t st = branch ? c->gstreams[gi] : c->cap;
    if (branch) cudaStreamWaitEvent(st, c->gevents[0], 0);
    for (size_t i = 0; i < gps[gi].size() && rc == SBI_OK; ++i, ++evi) {
      // external event records become timing nodes of the graph
      if (c->prof) cudaEventRecordWithFlags(ge.ev[2 * evi], st, cudaEventRecordExternal);
      rc = launch_pass(c, gps[gi][i], st);
      if (c->prof) cudaEventRecordWithFlags(ge.ev[2 * evi + 1], st, cudaEventRecordExternal);
    }
    if (branch) {
      cudaEventRecord(c->gevents[gi + 1], st);
      cudaStreamWaitEvent(c->cap, c->gevents[gi + 1], 0);
    }
  }
  // the simulation time of the next step (read by the wavemaker passes)
  if (rc == SBI_OK && c->wm_n > 0 && kind == SK_STEP && !only) {
    k_advance_time<<<1, 32, 0, c->cap>>>(c->d_time, dt);
    const cudaError_t el = cudaGetLastError();
    if (el != cudaSuccess) rc = cuda_fail(c, el, "kernel launch");
    else ++npasses;
  }
  cudaError_t e = cudaStreamEndCapture(c->cap, &ge.graph);
  auto drop = [&]() {
    for (auto ev : ge.ev) cudaEventDestroy(ev);
    ge.ev.clear();
    if (ge.graph) cudaGraphDestroy(ge.graph);
    ge.graph = nullptr;
  };
  if (rc) {
    drop();
    return rc;
  }
  if (e != cudaSuccess) {
    drop();
    return cuda_fail(c, e, "end capture");
  }
  e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
  if (e != cudaSuccess) {
    drop();
    return cuda_fail(c, e, "graph instantiate");
  }
  ge.launches = (int)npasses;
  return SBI_OK;
}

void destroy_graph(GraphEntry& ge) {
  if (ge.exec) cudaGraphExecDestroy(ge.exec);
  if (ge.graph) cudaGraphDestroy(ge.graph);
  for (auto e : ge.ev) cudaEventDestroy(e);
  ge.exec = nullptr;
  ge.graph = nullptr;
  ge.ev.clear();
}

// Device buffers a step reads before it writes them: the state, the working
// copies of the state (physical eta, mixed eta^ and phi^), the simulation
// time and the non-finite flag.  A copy of them lets the schedule candidates
// be timed on real steps and the state be put back exactly afterwards.
struct Snapshot {
  std::vector<std::pair<void*, size_t>> bufs;
  void* scratch = nullptr;
  size_t total = 0;
};

void snapshot_free(sbi_ctx* c, Snapshot& s) {
  if (!s.scratch) return;
  cudaStreamSynchronize(c->cap);
  if (c->opt.dev_free) c->opt.dev_free(s.scratch, c->opt.alloc_user);
  else cudaFree(s.scratch);
  s.scratch = nullptr;
}

// 1: taken; 0: not enough device memory (nothing to undo); < 0: CUDA error
int snapshot_take(sbi_ctx* c, Snapshot& s) {
  auto add = [&](void* p, size_t bytes) {
    if (p && bytes) s.bufs.push_back({p, bytes});
  };
  for (auto& g : c->groups) {
    const size_t np = g.phys_elems() * (size_t)g.n;
    const size_t nm = g.mixed_elems() * (size_t)g.n * 2 * c->real_size;
    add(g.eta0, np * 8);
    add(g.phi0, np * 8);
    add(g.eta_w, np * c->real_size);
    for (const char* name : {"eta_m", "phi_m"}) {
      auto it = g.mixed.find(name);
      if (it != g.mixed.end()) add(it->second, nm);
    }
  }
  add(c->d_time, c->d_time ? sizeof(double) : 0);
  add(c->d_flags, 64);
  for (auto& b : s.bufs) s.total += (b.second + 255) / 256 * 256;
  void* p = nullptr;
  if (c->opt.dev_alloc) p = c->opt.dev_alloc(s.total, c->opt.alloc_user);
  else if (cudaMalloc(&p, s.total) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return 0;
  s.scratch = p;
  size_t off = 0;
  for (auto& b : s.bufs) {
    if (cudaMemcpyAsync((char*)p + off, b.first, b.second, cudaMemcpyDeviceToDevice, c->cap) != cudaSuccess)
      return -1;
    off += (b.second + 255) / 256 * 256;
  }
  return 1;
}

int snapshot_restore(sbi_ctx* c, const Snapshot& s) {
  size_t off = 0;
  for (auto& b : s.bufs) {
    CK(cudaMemcpyAsync(b.first, (char*)s.scratch + off, b.second, cudaMemcpyDeviceToDevice, c->cap), "restore");
    off += (b.second + 255) / 256 * 256;
  }
  CK(cudaStreamSynchronize(c->cap), "restore");
  return SBI_OK;
}

std::string sched_desc(const sbi_ctx* c, const Sched& s) {
  std::string d = s.name + (s.serial ? " [serial]" : " [concurrent]") + " " + std::to_string(s.units.size()) + " units:";
  for (const Unit& u : s.units) {
    const Group& g = c->groups[u.group];
    d += " " + std::to_string(g.nx) + "x" + std::to_string(g.ny) + "[" + std::to_string(u.m0) + ":" +
         std::to_string(u.m1) + "]";
  }
  return d;
}

// Choose the step schedule (see the comment above pass_sliceable).
int choose_schedule(sbi_ctx* c, double dt, int kind) {
  if (c->sched_done) return SBI_OK;
  bool oom = false;
  std::vector<Sched> cands = sched_candidates(c, &oom);
  if (oom) return fail(c, SBI_ENOMEM, "device allocation failed while planning the step");
  if (c->opt.schedule != 0) {
    // a schedule named by the caller: nothing is timed
    const Sched s = forced_sched(c, &oom);
    if (oom) return fail(c, SBI_ENOMEM, "device allocation failed while planning the step");
    c->units = s.units;
    c->serial = s.serial;
    c->sched_done = true;
    c->sched_report = "forced " + sched_desc(c, s) + "\n";
    return SBI_OK;
  }
  c->units = cands[0].units;
  c->serial = cands[0].serial;
  if (c->prof) return SBI_OK;   // a profiled replay keeps the default until a plain step chooses
  c->sched_done = true;
  c->sched_report = "default " + sched_desc(c, cands[0]) + "\n";
  if (!c->opt.autotune || kind != SK_STEP || cands.size() < 2) return SBI_OK;
  Snapshot snap;
  const int taken = snapshot_take(c, snap);
  if (taken < 0) {
    snapshot_free(c, snap);
    return cuda_fail(c, cudaGetLastError(), "state copy");
  }
  if (taken == 0) {
    c->sched_report += "not timed: no device memory for a copy of the state\n";
    return SBI_OK;
  }
  if (!c->tune_ev[0]) {
    CK(cudaEventCreate(&c->tune_ev[0]), "event");
    CK(cudaEventCreate(&c->tune_ev[1]), "event");
  }
  std::vector<double> ms(cands.size(), -1.0);
  int rc = SBI_OK;
  for (size_t i = 0; i < cands.size() && rc == SBI_OK; ++i) {
    c->units = cands[i].units;
    c->serial = cands[i].serial;
    GraphEntry ge;
    rc = build_step_graph(c, dt, kind, nullptr, ge);
    if (rc) break;
    auto replay = [&]() { return cudaGraphLaunch(ge.exec, c->cap); };
    cudaError_t e = replay();   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[0], c->cap);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = replay();
    if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[1], c->cap);
    if (e == cudaSuccess) e = cudaEventSynchronize(c->tune_ev[1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, c->tune_ev[0], c->tune_ev[1]);
    destroy_graph(ge);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "schedule timing");
    else ms[i] = t / 3.0;
    if (rc == SBI_OK) rc = snapshot_restore(c, snap);
  }
  snapshot_free(c, snap);
  if (rc) return rc;
  size_t best = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (ms[i] < ms[best]) best = i;
  if (best != 0 && !(ms[best] < 0.97 * ms[0])) best = 0;
  c->units = cands[best].units;
  c->serial = cands[best].serial;
  c->sched_report.clear();
  for (size_t i = 0; i < cands.size(); ++i) {
    char t[64];
    snprintf(t, sizeof(t), "%.4f ms per step: ", ms[i]);
    c->sched_report += std::string(i == best ? "chosen " : (i == 0 ? "default " : "tried ")) + t +
                       sched_desc(c, cands[i]) + "\n";
  }
  if (best != 0) c->sched_report += "default " + sched_desc(c, cands[0]) + "\n";
  return SBI_OK;
}

int get_step_graph(sbi_ctx* c, double dt, GraphEntry** out, int kind = SK_STEP, const Unit* only = nullptr) {
  if (!c->sched_done) {
    const int rc = choose_schedule(c, dt, kind);
    if (rc) return rc;
    // graphs captured under an earlier (default) schedule are dropped
    if (c->sched_done) free_graphs(c);
  }
  for (auto& ge : c->graphs)
    if (ge.dt == dt && ge.prof == c->prof && ge.kind == kind && ge.group == (only ? only->group : -1) &&
        (!only || (ge.m0 == only->m0 && ge.m1 == only->m1))) {
      *out = &ge;
      return SBI_OK;
    }
  GraphEntry ge;
  const int rc = build_step_graph(c, dt, kind, only, ge);
  if (rc) return rc;
  c->graphs.push_back(ge);
  *out = &c->graphs.back();
  return SBI_OK;
}

// Launch a captured graph; a profiled graph's event pairs are read back and
// added to the per-family totals.
int launch_graph(sbi_ctx* c, GraphEntry* ge) {
  CK(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
  if (c->prof) {
    CK(cudaStreamSynchronize(c->stream), "profile sync");
    for (size_t q = 0; q < ge->ev_family.size(); ++q) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ge->ev[2 * q], ge->ev[2 * q + 1]), "event time");
      c->prof_ms[ge->ev_family[q]] += ms;
      c->prof_launches[ge->ev_family[q]] += 1;
    }
  }
  return SBI_OK;
}

int check_member(sbi_ctx* c, int member) {
  if (!c) return SBI_EINVAL;
  if (member < 0 || member >= c->nmembers) return fail(c, SBI_EINVAL, "member %d out of range", member);
  return SBI_OK;
}

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_to_real(const double* __restrict__ src, T* __restrict__ dst, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = T(src[i]);
}
template <typename T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = double(src[i]);
}

// Partial sums of eta and 1/2 (phi V + g eta^2) over fixed chunks of one
// member, each chunk reduced by one block in a fixed tree order.
// one state value as a double (hi + lo float pairs in the FP32 path)
template <bool DS>
__device__ __forceinline__ double state_value(const void* base, long long i) {
  if constexpr (!DS) {
    return reinterpret_cast<const double*>(base)[i];
  } else {
    const float2 v = reinterpret_cast<const float2*>(base)[i];
    return double(v.x) + double(v.y);
  }
}

template <typename T, bool DS>
__global__ void k_invariant_partials(const void* __restrict__ eta, const void* __restrict__ phi,
                                     const T* __restrict__ V, long long n, double g, int chunk,
                                     double* __restrict__ out) {
  __shared__ double sm[2][256];
  const long long base = (long long)blockIdx.x * chunk;
  double m = 0.0, e = 0.0;
  for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
    const long long q = base + i;
    if (q < n) {
      const double h = state_value<DS>(eta, q);
      m += h;
      e += 0.5 * (state_value<DS>(phi, q) * double(V[q]) + g * h * h);
    }
  }
  sm[0][threadIdx.x] = m;
  sm[1][threadIdx.x] = e;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sm[0][0];
    out[2 * blockIdx.x + 1] = sm[1][0];
  }
}

int run_diag(sbi_ctx* c, int gi, bool eulerian) {
  std::vector<Pass> ps;
  Planner pl{c, c->groups[gi]};
  pl.plan_diag(ps);
  pl.plan_sum_v(ps, eulerian);
  if (pl.oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  CK(cudaStreamSynchronize(c->cap), "sync");
  for (auto& p : ps) {
    int rc = tune_pass(c, p, c->stream);
    if (!rc) rc = launch_pass(c, p, c->stream);
    if (rc) return rc;
  }
  return SBI_OK;
}

int init_group(sbi_ctx* c, Group& g) {
  const size_t np = g.phys_elems() * g.n;
  g.eta0 = (double*)dalloc(c, np * 8);
  g.phi0 = (double*)dalloc(c, np * 8);
  g.acc_eta = (double*)dalloc(c, np * 8);
  g.acc_phi = (double*)dalloc(c, np * 8);
  g.eta_w = dalloc(c, np * c->real_size);
  g.Vphys = dalloc(c, np * c->real_size);
  g.wout = dalloc(c, np * c->real_size);
  g.out64 = (double*)dalloc(c, g.phys_elems() * 8);
  g.d_active = (int*)dalloc(c, (size_t)g.n * sizeof(int));
  if (c->opt.adapt_tol > 0.0) {
    g.d_conv = (int*)dalloc(c, (size_t)g.n * sizeof(int));
    g.d_orders = (int*)dalloc(c, (size_t)g.n * sizeof(int));
    g.d_notconv = (int*)dalloc(c, (size_t)g.n * sizeof(int));
    g.d_red = (double*)dalloc(c, (size_t)g.n * kConvBlocks * 2 * sizeof(double));
    if (!g.d_conv || !g.d_orders || !g.d_notconv || !g.d_red)
      return fail(c, SBI_ENOMEM, "device allocation failed");
  }
  if (!g.eta0 || !g.phi0 || !g.acc_eta || !g.acc_phi || !g.eta_w || !g.Vphys || !g.wout ||
      !g.out64 || !g.d_active)
    return fail(c, SBI_ENOMEM, "device allocation failed");
  return SBI_OK;
}

template <typename T>
std::vector<T> to_real(const std::vector<double>& v) {
  std::vector<T> r(v.size());
  for (size_t i = 0; i < v.size(); ++i) r[i] = T(v[i]);
  return r;
}

int upload_real(sbi_ctx* c, void* dst, const std::vector<double>& v, size_t offset_elems) {
  if (c->fp64) {
    CK(cudaMemcpyAsync((double*)dst + offset_elems, v.data(), v.size() * 8, cudaMemcpyHostToDevice, c->cap), "upload");
  } else {
    std::vector<float> f = to_real<float>(v);
    CK(cudaMemcpyAsync((float*)dst + offset_elems, f.data(), f.size() * 4, cudaMemcpyHostToDevice, c->cap), "upload");
    CK(cudaStreamSynchronize(c->cap), "upload sync");
  }
  CK(cudaStreamSynchronize(c->cap), "upload sync");
  return SBI_OK;
}

int create_impl(int n, const sbi_grid* grids, double gravity, const double* const* h,
                const sbi_options* opt_in, sbi_ctx** out) {
  if (!out) return fail(nullptr, SBI_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !grids) return fail(nullptr, SBI_EINVAL, "need at least one grid");
  sbi_options opt;
  sbi_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.order < 1 || opt.order > 7) return fail(nullptr, SBI_EINVAL, "order %d outside 1..7", opt.order);
  if (!(opt.alias_frac > 0.0 && opt.alias_frac <= 1.0))
    return fail(nullptr, SBI_EINVAL, "alias_frac must be in (0, 1]");
  if (!(gravity > 0.0) || !std::isfinite(gravity)) return fail(nullptr, SBI_EINVAL, "gravity must be > 0");
  if (opt.precision != SBI_FP32 && opt.precision != SBI_FP64)
    return fail(nullptr, SBI_EINVAL, "precision must be SBI_FP32 or SBI_FP64");
  if (opt.filt_beta1 > 0.0 && !(opt.k_ref > 0.0 && opt.filt_beta2 > 0.0))
    return fail(nullptr, SBI_EINVAL, "filter needs k_ref > 0 and beta2 > 0");
  if (opt.adapt_tol < 0.0) return fail(nullptr, SBI_EINVAL, "adapt_tol must be >= 0");
  if (opt.integrator != SBI_RK4 && opt.integrator != SBI_LAWSON_RK4 && opt.integrator != SBI_IF_RK45)
    return fail(nullptr, SBI_EINVAL, "integrator must be SBI_RK4, SBI_LAWSON_RK4 or SBI_IF_RK45");
  if (opt.diagnostic != SBI_DIAG_ESBI && opt.diagnostic != SBI_DIAG_HOS)
    return fail(nullptr, SBI_EINVAL, "diagnostic must be SBI_DIAG_ESBI or SBI_DIAG_HOS");
  if (opt.diagnostic == SBI_DIAG_HOS && opt.adapt_tol > 0.0)
    return fail(nullptr, SBI_EINVAL, "the HOS diagnostic is not combined with adapt_tol > 0");
  if (opt.integrator != SBI_RK4 && opt.adapt_tol > 0.0)
    return fail(nullptr, SBI_EINVAL, "the integrating factor (integrator) is not combined with adapt_tol > 0");
  if (opt.schedule < -1) return fail(nullptr, SBI_EINVAL, "schedule must be -1, 0 or a positive B");
  if (opt.col_staging < -1 || opt.col_staging > 1) return fail(nullptr, SBI_EINVAL, "col_staging must be -1, 0 or 1");
  if ((opt.dev_alloc == nullptr) != (opt.dev_free == nullptr))
    return fail(nullptr, SBI_EINVAL, "dev_alloc and dev_free must be given together");
  for (int i = 0; i < n; ++i) {
    const sbi_grid& g = grids[i];
    if (!is_pow2(g.nx) || g.nx < 16 || g.nx > 4096)
      return fail(nullptr, SBI_EINVAL, "grid %d: nx=%d must be a power of two in [16, 4096]", i, g.nx);
    if (!(g.ny == 1 || (is_pow2(g.ny) && g.ny >= 8 && g.ny <= 2048)))
      return fail(nullptr, SBI_EINVAL, "grid %d: ny=%d must be 1 or a power of two in [8, 2048]", i, g.ny);
    if (!(g.Lx > 0.0) || (g.ny > 1 && !(g.Ly > 0.0)))
      return fail(nullptr, SBI_EINVAL, "grid %d: box lengths must be > 0", i);
  }
  if (opt.sponge_w) {
    for (int i = 1; i < n; ++i)
      if (grids[i].nx != grids[0].nx || grids[i].ny != grids[0].ny)
        return fail(nullptr, SBI_EINVAL, "a sponge weight needs every member on one grid");
  }

  sbi_ctx* c = new sbi_ctx();
  c->opt = opt;
  c->gravity = gravity;
  c->fp64 = opt.precision == SBI_FP64;
  c->state_ds = !c->fp64 && !opt.state_fp64;
  c->real_size = c->fp64 ? 8 : 4;
  c->nmembers = n;
  c->stream = (cudaStream_t)opt.cuda_stream;
  auto bail = [&](int rc) {
    g_create_error = c->err;
    sbi_destroy(c);
    return rc;
  };
  // depth per member
  std::vector<double> h0s(n);
  std::vector<bool> var(n, false);
  std::vector<std::vector<double>> deltas(n);
  for (int i = 0; i < n; ++i) {
    const sbi_grid& g = grids[i];
    const size_t np = (size_t)g.nx * g.ny;
    const double* hi = h ? h[i] : nullptr;
    double h0 = opt.h0;
    if (!hi) {
      if (std::isnan(h0) || !(h0 > 0.0)) {
        c->err = "a flat member needs opt.h0 > 0 (or INFINITY)";
        return bail(SBI_EINVAL);
      }
    } else {
      double sum = 0.0;
      for (size_t q = 0; q < np; ++q) {
        if (!(hi[q] > 0.0) || !std::isfinite(hi[q])) {
          c->err = "depth h must be finite and > 0";
          return bail(SBI_EINVAL);
        }
        sum += hi[q];
      }
      if (std::isnan(h0)) h0 = sum / (double)np;
      if (!(h0 > 0.0) || !std::isfinite(h0)) {
        c->err = "reference depth h0 must be finite and > 0 with a depth field";
        return bail(SBI_EINVAL);
      }
      deltas[i].resize(np);
      for (size_t q = 0; q < np; ++q) {
        deltas[i][q] = h0 - hi[q];
        if (deltas[i][q] != 0.0) var[i] = true;
      }
    }
    h0s[i] = h0;
    if (var[i] && opt.diagnostic == SBI_DIAG_HOS) {
      c->err = "the HOS diagnostic needs a flat bottom (h == NULL or constant h)";
      return bail(SBI_EINVAL);
    }
  }

  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cannot create a CUDA stream (no usable device?)";
    return bail(SBI_ECUDA);
  }

  // group members with identical grids and depth settings: every pass of a
  // group is one launch over its members (or over a member range of it, see
  // the step schedule)
  c->where.resize(n);
  std::vector<int> sig(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < i && sig[i] < 0; ++j)
      if (grids[j].nx == grids[i].nx && grids[j].ny == grids[i].ny && grids[j].Lx == grids[i].Lx &&
          (grids[i].ny == 1 || grids[j].Ly == grids[i].Ly) && h0s[j] == h0s[i] && var[j] == var[i])
        sig[i] = sig[j];
    if (sig[i] < 0) {
      sig[i] = (int)c->groups.size();
      Group g;
      g.nx = grids[i].nx;
      g.ny = grids[i].ny;
      g.Lx = grids[i].Lx;
      g.Ly = grids[i].ny > 1 ? grids[i].Ly : 1.0;
      g.h0 = h0s[i];
      g.deep = std::isinf(h0s[i]);
      g.variable = var[i];
      g.two_d = g.ny > 1;
      const double A = opt.alias_frac * g.nx / 2.0, B = opt.alias_frac * g.ny / 2.0;
      g.kx_keep = std::min((int)std::ceil(A - 1e-12), g.nx / 2);
      g.ky_keep = g.ny == 1 ? 1 : std::min((int)std::ceil(B - 1e-12), g.ny / 2);
      g.kx_keep = std::max(g.kx_keep, 1);
      g.ky_keep = std::max(g.ky_keep, 1);
      g.W = g.kx_keep;
      c->groups.push_back(g);
    }
    Group& g = c->groups[sig[i]];
    c->where[i] = {sig[i], (int)g.members.size()};
    g.members.push_back(i);
  }
  for (auto& g : c->groups) g.n = (int)g.members.size();

  // twiddles exp(-2 pi i j / N) for N = 2..8192 in the working precision
  {
    const int tot = 8192 * 2 - 2;
    std::vector<double> re(tot), im(tot);
    for (int N = 2; N <= 8192; N *= 2)
      for (int j = 0; j < N; ++j) {
        const double a = -2.0 * M_PI * (double)j / (double)N;
        re[N - 2 + j] = std::cos(a);
        im[N - 2 + j] = std::sin(a);
      }
    c->tw = dalloc(c, (size_t)tot * 2 * c->real_size);
    if (!c->tw) { c->err = "device allocation failed"; return bail(SBI_ENOMEM); }
    std::vector<double> inter(2 * (size_t)tot);
    for (int q = 0; q < tot; ++q) { inter[2 * q] = re[q]; inter[2 * q + 1] = im[q]; }
    if (upload_real(c, c->tw, inter, 0)) return bail(SBI_ECUDA);
  }
  c->d_flags = (int*)dalloc(c, 64);
  if (!c->d_flags) { c->err = "device allocation failed"; return bail(SBI_ENOMEM); }

  for (auto& g : c->groups) {
    cudaError_t e = c->fp64 ? prepare_row_kernels<double>(g.nx) : prepare_row_kernels<float>(g.nx);
    if (e == cudaSuccess) e = c->fp64 ? prepare_col_kernels<double>(g.ny) : prepare_col_kernels<float>(g.ny);
    if (e != cudaSuccess) { cuda_fail(c, e, "kernel setup"); return bail(SBI_ECUDA); }
    int rc = init_group(c, g);
    if (rc) return bail(rc);
    if (g.variable) {
      g.delta = dalloc(c, g.phys_elems() * g.n * c->real_size);
      if (!g.delta) { c->err = "device allocation failed"; return bail(SBI_ENOMEM); }
    }
  }
  // bathymetry
  for (int i = 0; i < n; ++i) {
    Group& g = c->groups[c->where[i].first];
    if (g.variable) {
      if (upload_real(c, g.delta, deltas[i], (size_t)c->where[i].second * g.phys_elems()))
        return bail(SBI_ECUDA);
    }
  }
  if (opt.sponge_w && opt.sponge_nu != 0.0) {
    const size_t np = (size_t)grids[0].nx * grids[0].ny;
    std::vector<double> w(opt.sponge_w, opt.sponge_w + np);
    c->wgt = dalloc(c, np * c->real_size);
    if (!c->wgt) { c->err = "device allocation failed"; return bail(SBI_ENOMEM); }
    if (upload_real(c, c->wgt, w, 0)) return bail(SBI_ECUDA);
  }
  c->opt.sponge_w = nullptr;  // the host array is not kept
  c->orders_used.assign(n, opt.order);
  // working copies of the zero state
  for (auto& g : c->groups) {
    Planner pl{c, g};
    std::vector<Pass> ps;
    ps.push_back(pl.plan_rk(RK_ENTRY, 0, 0.0, 1));
    if (pl.oom) { c->err = "device allocation failed"; return bail(SBI_ENOMEM); }
    if (run_passes(c, ps, c->cap)) return bail(SBI_ECUDA);
  }
  if (cudaStreamSynchronize(c->cap) != cudaSuccess) {
    cuda_fail(c, cudaGetLastError(), "create");
    return bail(SBI_ECUDA);
  }
  *out = c;
  return SBI_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void sbi_default_options(sbi_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->order = 7;
  opt->alias_frac = 0.5;
  opt->h0 = NAN;
  opt->precision = SBI_FP32;
  opt->state_fp64 = 0;
  opt->adapt_tol = 0.0;
  opt->filt_beta1 = 0.0;
  opt->filt_beta2 = 0.0;
  opt->k_ref = 1.0;
  opt->sponge_w = nullptr;
  opt->sponge_nu = 0.0;
  opt->cuda_stream = nullptr;
  opt->check_finite = 1;
  opt->set_state_dealias = 1;
  opt->autotune = 1;
  opt->schedule = 0;
  opt->col_staging = 0;
}

int sbi_create(const sbi_grid* g, double gravity, const double* h, const sbi_options* opt,
               sbi_ctx** out) {
  if (!g) return fail(nullptr, SBI_EINVAL, "grid is NULL");
  const double* hs[1] = {h};
  return create_impl(1, g, gravity, hs, opt, out);
}

int sbi_create_batch(int n, const sbi_grid* grids, double gravity, const double* const* h,
                     const sbi_options* opt, sbi_ctx** out) {
  return create_impl(n, grids, gravity, h, opt, out);
}

int sbi_num_members(const sbi_ctx* ctx) { return ctx ? ctx->nmembers : 0; }

int sbi_set_state(sbi_ctx* c, int member, const double* eta, const double* phi, int on_device) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!eta || !phi) return fail(c, SBI_EINVAL, "eta and phi must not be NULL");
  Group& g = c->groups[c->where[member].first];
  const size_t off = (size_t)c->where[member].second * g.phys_elems();
  const long long np = (long long)g.phys_elems();
  CK(cudaStreamSynchronize(c->stream), "sync");
  const double* srcs[2] = {eta, phi};
  double* dsts[2] = {g.eta0 + off, g.phi0 + off};
  for (int q = 0; q < 2; ++q) {
    const double* src = srcs[q];
    if (!on_device) {
      CK(cudaMemcpyAsync(g.out64, srcs[q], np * 8, cudaMemcpyHostToDevice, c->cap), "copy state");
      src = g.out64;
    }
    cudaError_t e = !c->state_ds ? state_convert<double>(src, dsts[q], np, false, c->cap)
                            : state_convert<float>(src, dsts[q], np, false, c->cap);
    CK(e, "state conversion");
  }
  // dealias the stored state of this member only: (M - 1) correction; then
  // refresh this member's working copies
  std::vector<int> act(g.n, 0);
  act[c->where[member].second] = 1;
  CK(cudaMemcpyAsync(g.d_active, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, c->cap), "active");
  Planner pl{c, g};
  std::vector<Pass> ps;
  if (c->opt.set_state_dealias) pl.plan_project(ps, false);
  else ps.push_back(pl.plan_rk(RK_ENTRY, 0, 0.0, 1));
  if (pl.oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  for (auto& p : ps) {
    if (p.kind == PK_ROW) p.row.active = g.d_active;
    else if (p.kind == PK_COL) p.col.active = g.d_active;
    else p.rk.active = g.d_active;
  }
  rc = run_passes(c, ps, c->cap);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->cap), "set_state");
  return SBI_OK;
}

// offset (in doubles) of each member's field in a concatenated buffer
std::vector<size_t> member_offsets(const sbi_ctx* c) {
  std::vector<size_t> off(c->nmembers + 1, 0);
  for (int m = 0; m < c->nmembers; ++m) {
    const Group& g = c->groups[c->where[m].first];
    off[m + 1] = off[m] + g.phys_elems();
  }
  return off;
}

// The device address of a caller's buffer that kernels can read and write
// directly: device memory (on_device), or host memory that is pinned and
// mapped (on this system it is reached over the host link); nullptr when the
// buffer must go through a copy.
double* device_view(void* p, int on_device) {
  if (on_device) return static_cast<double*>(p);
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<double*>(a.devicePointer);
  return nullptr;
}

int ensure_stage(sbi_ctx* c, Group& g) {
  if (!g.stage64) g.stage64 = (double*)dalloc(c, g.phys_elems() * g.n * 8);
  return g.stage64 ? SBI_OK : fail(c, SBI_ENOMEM, "device allocation failed");
}

int sbi_set_state_all(sbi_ctx* c, const double* eta, const double* phi, int on_device) {
  if (!c) return SBI_EINVAL;
  if (!eta || !phi) return fail(c, SBI_EINVAL, "eta and phi must not be NULL");
  const std::vector<size_t> off = member_offsets(c);
  CK(cudaStreamSynchronize(c->stream), "sync");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* srcs[2] = {eta, phi};
  const double* views[2] = {device_view(const_cast<double*>(eta), on_device),
                            device_view(const_cast<double*>(phi), on_device)};
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    Group& g = c->groups[gi];
    const size_t np = g.phys_elems();
    double* dsts[2] = {g.eta0, g.phi0};
    for (int q = 0; q < 2; ++q) {
      // per run of members that are consecutive in the caller's buffer: the
      // conversion kernel reads the caller's buffer itself when it can, else
      // the run is copied into the staging buffer and converted from there
      if (!views[q]) {
        int rc = ensure_stage(c, g);
        if (rc) return rc;
      }
      for (int li = 0; li < g.n;) {
        int run = 1;
        while (li + run < g.n && g.members[li + run] == g.members[li] + run) ++run;
        const double* from = views[q] ? views[q] + off[g.members[li]] : g.stage64 + (size_t)li * np;
        if (!views[q])
          CK(cudaMemcpyAsync(g.stage64 + (size_t)li * np, srcs[q] + off[g.members[li]], np * 8 * run,
                             kind, c->cap), "copy state");
        void* to = reinterpret_cast<char*>(dsts[q]) + (size_t)li * np * 8;   // 8 bytes per stored value
        cudaError_t e = !c->state_ds ? state_convert<double>(from, to, (long long)(np * run), false, c->cap)
                                : state_convert<float>(from, to, (long long)(np * run), false, c->cap);
        CK(e, "state conversion");
        li += run;
      }
    }
    // dealias (or only refresh the working copies of) every member of the group
    Planner pl{c, g};
    std::vector<Pass> ps;
    if (c->opt.set_state_dealias) pl.plan_project(ps, false);
    else ps.push_back(pl.plan_rk(RK_ENTRY, 0, 0.0, 1));
    if (pl.oom) return fail(c, SBI_ENOMEM, "device allocation failed");
    const int rc = run_passes(c, ps, c->cap);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->cap), "set_state_all");
  return SBI_OK;
}

int sbi_get_state_all(sbi_ctx* c, double* eta, double* phi, int on_device) {
  if (!c) return SBI_EINVAL;
  if (!eta || !phi) return fail(c, SBI_EINVAL, "eta and phi must not be NULL");
  const std::vector<size_t> off = member_offsets(c);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dsts[2] = {eta, phi};
  double* views[2] = {device_view(eta, on_device), device_view(phi, on_device)};
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    Group& g = c->groups[gi];
    const size_t np = g.phys_elems();
    const double* srcs[2] = {g.eta0, g.phi0};
    for (int q = 0; q < 2; ++q) {
      if (views[q]) {
        // the conversion kernel writes the caller's buffer itself, one
        // launch per run of consecutive members
        for (int li = 0; li < g.n;) {
          int run = 1;
          while (li + run < g.n && g.members[li + run] == g.members[li] + run) ++run;
          const void* from = reinterpret_cast<const char*>(srcs[q]) + (size_t)li * np * 8;
          cudaError_t e = !c->state_ds
              ? state_convert<double>(from, views[q] + off[g.members[li]], (long long)(np * run), true, c->stream)
              : state_convert<float>(from, views[q] + off[g.members[li]], (long long)(np * run), true, c->stream);
          CK(e, "state conversion");
          li += run;
        }
        continue;
      }
      int rc = ensure_stage(c, g);
      if (rc) return rc;
      cudaError_t e = !c->state_ds ? state_convert<double>(srcs[q], g.stage64, (long long)(np * g.n), true, c->stream)
                              : state_convert<float>(srcs[q], g.stage64, (long long)(np * g.n), true, c->stream);
      CK(e, "state conversion");
      for (int li = 0; li < g.n;) {   // one copy per run of consecutive members
        int run = 1;
        while (li + run < g.n && g.members[li + run] == g.members[li] + run) ++run;
        CK(cudaMemcpyAsync(dsts[q] + off[g.members[li]], g.stage64 + (size_t)li * np, np * 8 * run,
                           kind, c->stream), "copy state");
        li += run;
      }
    }
  }
  CK(cudaStreamSynchronize(c->stream), "get_state_all");
  return SBI_OK;
}

int sbi_get_state(sbi_ctx* c, int member, double* eta, double* phi, int on_device) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!eta || !phi) return fail(c, SBI_EINVAL, "eta and phi must not be NULL");
  Group& g = c->groups[c->where[member].first];
  const size_t off = (size_t)c->where[member].second * g.phys_elems();
  const long long np = (long long)g.phys_elems();
  const double* srcs[2] = {g.eta0 + off, g.phi0 + off};
  double* dsts[2] = {eta, phi};
  for (int q = 0; q < 2; ++q) {
    double* dst = on_device ? dsts[q] : g.out64;
    cudaError_t e = !c->state_ds ? state_convert<double>(srcs[q], dst, np, true, c->stream)
                            : state_convert<float>(srcs[q], dst, np, true, c->stream);
    CK(e, "state conversion");
    if (!on_device)
      CK(cudaMemcpyAsync(dsts[q], g.out64, np * 8, cudaMemcpyDeviceToHost, c->stream), "copy state");
  }
  CK(cudaStreamSynchronize(c->stream), "get_state");
  return SBI_OK;
}

// one member's physical field of the working precision -> FP64 V_out
// (host or device), queued on the library's stream
int output_member_field(sbi_ctx* c, int member, const void* src, double* V_out, int on_device) {
  Group& g = c->groups[c->where[member].first];
  const size_t np = g.phys_elems();
  const size_t off = (size_t)c->where[member].second * np;
  double* dst = on_device ? V_out : g.out64;
  const int thr = 256;
  const long long blocks = ((long long)np + thr - 1) / thr;
  if (c->fp64) k_to_double<double><<<(unsigned)blocks, thr, 0, c->stream>>>((const double*)src + off, dst, (long long)np);
  else k_to_double<float><<<(unsigned)blocks, thr, 0, c->stream>>>((const float*)src + off, dst, (long long)np);
  CK(cudaGetLastError(), "convert");
  if (!on_device)
    CK(cudaMemcpyAsync(V_out, g.out64, np * 8, cudaMemcpyDeviceToHost, c->stream), "copy V");
  return SBI_OK;
}

int sbi_vertical_velocity(sbi_ctx* c, int member, double* V_out, int on_device, int eulerian_w) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!V_out) return fail(c, SBI_EINVAL, "V_out is NULL");
  const int gi = c->where[member].first;
  Group& g = c->groups[gi];
  rc = run_diag(c, gi, eulerian_w != 0);
  if (rc) return rc;
  rc = output_member_field(c, member, eulerian_w ? g.wout : g.Vphys, V_out, on_device);
  if (rc) return rc;
  int notconv = 0;
  if (g.d_notconv)
    CK(cudaMemcpyAsync(&notconv, g.d_notconv + c->where[member].second, sizeof(int),
                       cudaMemcpyDeviceToHost, c->stream), "flag");
  CK(cudaStreamSynchronize(c->stream), "vertical_velocity");
  if (notconv)
    return fail(c, SBI_ENOTCONVERGED, "adaptive order reached %d without meeting adapt_tol "
                "(V is the order-%d sum)", c->opt.order, c->opt.order);
  return SBI_OK;
}

int sbi_crest(sbi_ctx* c, int member, double* x, double* y, double* height) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!x || !y || !height) return fail(c, SBI_EINVAL, "x, y and height must not be NULL");
  Group& g = c->groups[c->where[member].first];
  const size_t np = g.phys_elems();
  const size_t off = (size_t)c->where[member].second * np;
  if (!g.d_crest) {
    g.d_crest = (double*)dalloc(c, 3 * sizeof(double));
    if (!g.d_crest) return fail(c, SBI_ENOMEM, "device allocation failed");
    CK(cudaStreamSynchronize(c->cap), "sync");
  }
  cudaError_t e = !c->state_ds ? state_convert<double>(g.eta0 + off, g.out64, (long long)np, true, c->stream)
                          : state_convert<float>(g.eta0 + off, g.out64, (long long)np, true, c->stream);
  CK(e, "state conversion");
  k_crest<<<1, 256, 0, c->stream>>>(g.out64, g.nx, g.ny, g.Lx / g.nx, g.two_d ? g.Ly / g.ny : 0.0, g.d_crest);
  CK(cudaGetLastError(), "crest");
  double h[3];
  CK(cudaMemcpyAsync(h, g.d_crest, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy crest");
  CK(cudaStreamSynchronize(c->stream), "crest");
  *x = h[0];
  *y = h[1];
  *height = h[2];
  return SBI_OK;
}

int sbi_vertical_velocity_implicit(sbi_ctx* c, int member, int iterations, double* V_out, int on_device,
                                   double* increments) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!V_out) return fail(c, SBI_EINVAL, "V_out is NULL");
  if (iterations < 1 || iterations > kImplicitMaxIter)
    return fail(c, SBI_EINVAL, "iterations must be in 1..%d", kImplicitMaxIter);
  const int gi = c->where[member].first;
  Group& g = c->groups[gi];
  Planner pl{c, g};
  std::vector<Pass> setup, first, ab, ba, fin;
  if (g.variable) {
    // V and grad varphi~ iterated together (Appendices A and B)
    pl.plan_implicit_setup_var(setup);
    pl.plan_implicit_iter_var(first, "V1", "db1x", "db1y", "IVa", "IBxa", "IBya");
    pl.plan_implicit_iter_var(ab, "IVa", "IBxa", "IBya", "IVb", "IBxb", "IByb");
    pl.plan_implicit_iter_var(ba, "IVb", "IBxb", "IByb", "IVa", "IBxa", "IBya");
  } else {
    pl.plan_implicit_setup(setup);
    pl.plan_implicit_iter(first, "V1", "IVa");
    pl.plan_implicit_iter(ab, "IVa", "IVb");
    pl.plan_implicit_iter(ba, "IVb", "IVa");
  }
  const char* last = (iterations % 2) ? "IVa" : "IVb";
  {
    Planner::RowB r = pl.row_begin();
    pl.c2r(r, 0, {last}, g.Vphys);
    fin.push_back(pl.row_end(r, false, false, false));
  }
  if (!g.d_implicit)
    g.d_implicit = (double*)dalloc(c, (size_t)kImplicitMaxIter * g.n * 2 * sizeof(double));
  if (pl.oom || !g.d_implicit) return fail(c, SBI_ENOMEM, "device allocation failed");
  CK(cudaStreamSynchronize(c->cap), "sync");
  auto run = [&](std::vector<Pass>& v) {
    for (auto& p : v) {
      int r2 = tune_pass(c, p, c->stream);
      if (!r2) r2 = launch_pass(c, p, c->stream);
      if (r2) return r2;
    }
    return (int)SBI_OK;
  };
  rc = run(setup);
  if (rc) return rc;
  const long long stride = (long long)g.mixed_elems();
  for (int it = 0; it < iterations; ++it) {
    rc = run(it == 0 ? first : (it % 2 ? ab : ba));
    if (rc) return rc;
    const void* dst = pl.mixed(it % 2 ? "IVb" : "IVa");
    const void* src = pl.mixed(it == 0 ? "V1" : (it % 2 ? "IVa" : "IVb"));
    double* out = g.d_implicit + (size_t)it * g.n * 2;
    if (c->fp64) k_implicit_norms<double><<<g.n, 256, 0, c->stream>>>(dst, src, stride, g.W, g.ny, out);
    else k_implicit_norms<float><<<g.n, 256, 0, c->stream>>>(dst, src, stride, g.W, g.ny, out);
    CK(cudaGetLastError(), "implicit norms");
  }
  rc = run(fin);
  if (rc) return rc;
  rc = output_member_field(c, member, g.Vphys, V_out, on_device);
  if (rc) return rc;
  std::vector<double> nrm((size_t)iterations * g.n * 2);
  CK(cudaMemcpyAsync(nrm.data(), g.d_implicit, nrm.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "copy norms");
  CK(cudaStreamSynchronize(c->stream), "vertical_velocity_implicit");
  if (increments) {
    const int li = c->where[member].second;
    for (int it = 0; it < iterations; ++it) {
      const double d2 = nrm[((size_t)it * g.n + li) * 2], a2 = nrm[((size_t)it * g.n + li) * 2 + 1];
      increments[it] = a2 > 0.0 ? std::sqrt(d2 / a2) : 0.0;
    }
  }
  return SBI_OK;
}

// The device flags after a step: [0] the state became non-finite, [1] a
// bounded wait of a staged column pass gave up (cleared once reported).
int check_flags(sbi_ctx* c, const char* what) {
  int flag[2] = {0, 0};
  CK(cudaMemcpyAsync(flag, c->d_flags, sizeof(flag), cudaMemcpyDeviceToHost, c->stream), "flag");
  CK(cudaStreamSynchronize(c->stream), what);
  if (flag[1]) {
    CK(cudaMemsetAsync(c->d_flags + 1, 0, sizeof(int), c->stream), "flag");
    CK(cudaStreamSynchronize(c->stream), what);
    return fail(c, SBI_ETIMEOUT, "a bounded wait for a bulk copy of a column pass gave up");
  }
  if (flag[0]) return fail(c, SBI_ENONFINITE, "the state became non-finite");
  return SBI_OK;
}

int sbi_step(sbi_ctx* c, double dt, int n) {
  if (!c) return SBI_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SBI_EINVAL, "dt must be finite and > 0");
  if (n < 0) return fail(c, SBI_EINVAL, "n must be >= 0");
  if (n == 0) return SBI_OK;
  GraphEntry* ge = nullptr;
  int rc = SBI_OK;
  if (c->opt.integrator == SBI_IF_RK45) {
    // fixed steps of the adaptive scheme: the order-5 solution, the error
    // estimate not used
    GraphEntry *ga = nullptr, *gb = nullptr;
    rc = get_step_graph(c, 0.0, &ga, SK_RK45_A);
    if (!rc) rc = get_step_graph(c, 0.0, &gb, SK_RK45_B);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
      rc = update_dyn_tables(c, dt, c->stream);
      if (!rc) rc = launch_graph(c, ga);
      if (!rc) rc = launch_graph(c, gb);
      if (rc) return rc;
      c->t_host += dt;
    }
  } else {
    rc = get_step_graph(c, dt, &ge);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
      rc = launch_graph(c, ge);
      if (rc) return rc;
      c->t_host += dt;
    }
  }
  if (c->opt.check_finite) return check_flags(c, "step");
  return SBI_OK;
}

// Enqueue the upload, n steps and download of every member's state, one
// stream per unit (no synchronisation; the caller's stream waits for all).
int streamed_run(sbi_ctx* c, const double* eta_in, const double* phi_in, double dt, int n, double* eta_out,
                 double* phi_out, const std::vector<Unit>& units) {
  const size_t U = units.size();
  const std::vector<size_t> off = member_offsets(c);
  // everything that allocates, plans, tunes or synchronizes comes first
  std::vector<GraphEntry*> ges(U, nullptr);
  std::vector<std::vector<Pass>> entry(U);
  for (size_t ui = 0; ui < U; ++ui) {
    const Unit& u = units[ui];
    Group& g = c->groups[u.group];
    if (n > 0) {
      const int rc = get_step_graph(c, dt, &ges[ui], SK_STEP, &units[ui]);
      if (rc) return rc;
    }
    int rc = ensure_stage(c, g);
    if (rc) return rc;
    if (!g.stage64b) g.stage64b = (double*)dalloc(c, g.phys_elems() * g.n * 8);
    if (!g.stage64b) return fail(c, SBI_ENOMEM, "device allocation failed");
    Planner pl{c, g};
    std::vector<Pass> ps;
    if (c->opt.set_state_dealias) pl.plan_project(ps, false);
    else ps.push_back(pl.plan_rk(RK_ENTRY, 0, 0.0, 1));
    if (pl.oom) return fail(c, SBI_ENOMEM, "device allocation failed");
    for (const Pass& p : ps) entry[ui].push_back(slice_pass(p, g, u.m0, u.m1));
  }
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
  while (c->pstreams.size() < U) {
    cudaStream_t s2;
    const int prio = std::min(least, greatest + (int)c->pstreams.size());
    CK(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio), "stream");
    c->pstreams.push_back(s2);
  }
  while (c->pevents.size() < U + 1) {
    cudaEvent_t e2;
    CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "event");
    c->pevents.push_back(e2);
  }
  CK(cudaEventRecord(c->pevents[0], c->stream), "event");   // after the caller's earlier work
  const double* in[2] = {eta_in, phi_in};
  double* outp[2] = {eta_out, phi_out};
  // runs of members of a unit that are consecutive in the caller's buffers
  auto for_runs = [&](const Unit& u, const Group& g, auto&& f) -> int {
    for (int li = u.m0; li < u.m1;) {
      int run = 1;
      while (li + run < u.m1 && g.members[li + run] == g.members[li] + run) ++run;
      const int rc = f(li, run);
      if (rc) return rc;
      li += run;
    }
    return SBI_OK;
  };
  for (size_t ui = 0; ui < U; ++ui) {
    const Unit& u = units[ui];
    Group& g = c->groups[u.group];
    cudaStream_t st = c->pstreams[ui];
    const size_t np = g.phys_elems();
    const size_t first = (size_t)u.m0 * np, cnt = (size_t)(u.m1 - u.m0) * np;
    double* stage[2] = {g.stage64, g.stage64b};
    char* state[2] = {reinterpret_cast<char*>(g.eta0), reinterpret_cast<char*>(g.phi0)};
    CK(cudaStreamWaitEvent(st, c->pevents[0], 0), "wait");
    for (int q = 0; q < 2; ++q) {
      int rc = for_runs(u, g, [&](int li, int run) -> int {
        CK(cudaMemcpyAsync(stage[q] + (size_t)li * np, in[q] + off[g.members[li]], np * 8 * run,
                           cudaMemcpyDefault, st), "copy state");
        return SBI_OK;
      });
      if (rc) return rc;
      void* to = state[q] + first * 8;   // 8 bytes per stored value
      const cudaError_t e = !c->state_ds ? state_convert<double>(stage[q] + first, to, (long long)cnt, false, st)
                                         : state_convert<float>(stage[q] + first, to, (long long)cnt, false, st);
      CK(e, "state conversion");
    }
    int rc = run_passes(c, entry[ui], st);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(ges[ui]->exec, st), "graph launch");
    for (int q = 0; q < 2; ++q) {
      const void* from = state[q] + first * 8;
      const cudaError_t e = !c->state_ds ? state_convert<double>(from, stage[q] + first, (long long)cnt, true, st)
                                         : state_convert<float>(from, stage[q] + first, (long long)cnt, true, st);
      CK(e, "state conversion");
    }
  }
  // the downloads are queued after every unit's work: a copy into pageable
  // memory returns only when it is done and would hold back the next unit
  for (size_t ui = 0; ui < U; ++ui) {
    const Unit& u = units[ui];
    Group& g = c->groups[u.group];
    cudaStream_t st = c->pstreams[ui];
    const size_t np = g.phys_elems();
    double* stage[2] = {g.stage64, g.stage64b};
    for (int q = 0; q < 2; ++q) {
      const int rc = for_runs(u, g, [&](int li, int run) -> int {
        CK(cudaMemcpyAsync(outp[q] + off[g.members[li]], stage[q] + (size_t)li * np, np * 8 * run,
                           cudaMemcpyDefault, st), "copy state");
        return SBI_OK;
      });
      if (rc) return rc;
    }
    CK(cudaEventRecord(c->pevents[ui + 1], st), "event");
    CK(cudaStreamWaitEvent(c->stream, c->pevents[ui + 1], 0), "wait");
  }
  return SBI_OK;
}

// do [a, a + n) and [b, b + m) doubles overlap
bool overlaps(const double* a, size_t n, const double* b, size_t m) {
  const uintptr_t a0 = (uintptr_t)a, a1 = a0 + n * 8, b0 = (uintptr_t)b, b1 = b0 + m * 8;
  return a0 < b1 && b0 < a1;
}

// Upload, n steps and download of every member's state, pipelined per unit:
// each unit (a member range of one group) runs on its own stream (priority
// falling with the unit index), so the copies of one unit overlap the steps
// of the others.  The units are the step schedule's, each cut into k member
// ranges; smaller units start computing and finish copying out sooner, more
// of them make smaller launches.  On the first call (with autotuning, n > 0
// and outputs that overlap no input) k = 1, 2, 3, 4 and 6 are timed on whole
// one-step calls (each writes the outputs, which the call itself then
// overwrites) and the fastest is kept; k = 1 stays unless another is 3 %
// faster.  Every launch and its arguments are those of sbi_set_state_all +
// sbi_step + sbi_get_state_all restricted to a unit's members (same passes,
// same block shapes), so the result is the same bits for every k.
int sbi_step_streamed(sbi_ctx* c, const double* eta_in, const double* phi_in, double dt, int n,
                      double* eta_out, double* phi_out) {
  if (!c) return SBI_EINVAL;
  if (!eta_in || !phi_in || !eta_out || !phi_out) return fail(c, SBI_EINVAL, "state buffers must not be NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SBI_EINVAL, "dt must be finite and > 0");
  if (n < 0) return fail(c, SBI_EINVAL, "n must be >= 0");
  auto three_calls = [&]() {
    int rc = sbi_set_state_all(c, eta_in, phi_in, 0);
    if (!rc) rc = sbi_step(c, dt, n);
    if (!rc) rc = sbi_get_state_all(c, eta_out, phi_out, 0);
    return rc;
  };
  // the adaptive pair (host-side tables per step), the wavemaker (one clock
  // for every group) and profiling keep the three calls in order
  if (c->opt.integrator == SBI_IF_RK45 || c->wm_n > 0 || c->prof) return three_calls();
  // the schedule is chosen (and the whole-batch graph captured) first
  if (n > 0) {
    GraphEntry* ge_all = nullptr;
    const int rc = get_step_graph(c, dt, &ge_all);
    if (rc) return rc;
  } else if (c->units.empty()) {
    bool oom = false;
    plan_step_units(c, dt, &oom);
    if (oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  }
  const std::vector<Unit> units = c->units;
  if (units.size() < 2) return three_calls();
  if (c->stream_k == 0) {
    size_t total = 0;
    for (const auto& g : c->groups) total += g.phys_elems() * (size_t)g.n;
    const bool alias = overlaps(eta_in, total, eta_out, total) || overlaps(eta_in, total, phi_out, total) ||
                       overlaps(phi_in, total, eta_out, total) || overlaps(phi_in, total, phi_out, total);
    std::vector<int> ks = {1};
    for (int k : {2, 3, 4, 6})
      if (split_units(units, k).size() > split_units(units, ks.back()).size()) ks.push_back(k);
    if (!c->opt.autotune || n == 0 || alias || ks.size() < 2) {
      if (n > 0 || !c->opt.autotune) c->stream_k = 1;
    } else {
      if (!c->tune_ev[0]) {
        CK(cudaEventCreate(&c->tune_ev[0]), "event");
        CK(cudaEventCreate(&c->tune_ev[1]), "event");
      }
      std::vector<double> ms(ks.size(), -1.0);
      for (size_t i = 0; i < ks.size(); ++i) {
        const std::vector<Unit> su = split_units(units, ks[i]);
        int rc = streamed_run(c, eta_in, phi_in, dt, 1, eta_out, phi_out, su);   // warm-up
        if (rc) return rc;
        CK(cudaStreamSynchronize(c->stream), "streamed timing");
        CK(cudaEventRecord(c->tune_ev[0], c->stream), "event");
        rc = streamed_run(c, eta_in, phi_in, dt, 1, eta_out, phi_out, su);
        if (rc) return rc;
        CK(cudaEventRecord(c->tune_ev[1], c->stream), "event");
        CK(cudaEventSynchronize(c->tune_ev[1]), "streamed timing");
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->tune_ev[0], c->tune_ev[1]), "event time");
        ms[i] = t;
      }
      size_t best = 0;
      for (size_t i = 1; i < ks.size(); ++i)
        if (ms[i] < ms[best]) best = i;
      if (best != 0 && !(ms[best] < 0.97 * ms[0])) best = 0;
      c->stream_k = ks[best];
      for (size_t i = 0; i < ks.size(); ++i) {
        const std::vector<Unit> su = split_units(units, ks[i]);
        char t[96];
        snprintf(t, sizeof(t), "%s %.4f ms per step: ", i == best ? "streamed-chosen" : "streamed-tried", ms[i]);
        c->sched_report += std::string(t) +
                           sched_desc(c, Sched{su, false, "streamed split x" + std::to_string(ks[i])}) + "\n";
      }
    }
  }
  const std::vector<Unit> su = split_units(units, std::max(1, c->stream_k));
  const int rc = streamed_run(c, eta_in, phi_in, dt, n, eta_out, phi_out, su);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) c->t_host += dt;
  CK(cudaStreamSynchronize(c->stream), "step_streamed");
  if (c->opt.check_finite && n > 0) return check_flags(c, "step_streamed");
  return SBI_OK;
}

// The step after an error err at step h (the controller of the adaptive
// integrating factor).
double next_step_size(double h, double err, double tol) {
  if (err == 0.0) return 5.0 * h;
  return h * std::min(5.0, std::max(0.2, 0.9 * std::pow(tol / err, 0.2)));
}

int sbi_step_adaptive(sbi_ctx* c, double t_end, double tol, double* h_inout, int* accepted,
                      int* rejected) {
  if (!c) return SBI_EINVAL;
  if (c->opt.integrator != SBI_IF_RK45)
    return fail(c, SBI_EINVAL, "sbi_step_adaptive needs integrator = SBI_IF_RK45");
  if (!h_inout || !(*h_inout > 0.0) || !std::isfinite(*h_inout))
    return fail(c, SBI_EINVAL, "the initial step must be finite and > 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(c, SBI_EINVAL, "tol must be finite and > 0");
  if (!std::isfinite(t_end)) return fail(c, SBI_EINVAL, "t_end must be finite");
  GraphEntry *ga = nullptr, *gb = nullptr;
  int rc = get_step_graph(c, 0.0, &ga, SK_RK45_A);
  if (!rc) rc = get_step_graph(c, 0.0, &gb, SK_RK45_B);
  if (rc) return rc;
  double t = c->t_host, h = *h_inout;
  const double span = t_end - t;
  int acc = 0, rej = 0;
  std::vector<double> nrm;
  while (t < t_end) {
    const bool last = t + h >= t_end;
    const double hh = last ? t_end - t : h;
    rc = update_dyn_tables(c, hh, c->stream);
    if (!rc) rc = launch_graph(c, ga);
    if (rc) return rc;
    // error: max over members and fields of ||u5 - u4|| / ||u_n||; the offsets
    // are normalised for the inverse row transform, u_n's spectra are not
    // (factor nx)
    double err = 0.0;
    for (auto& g : c->groups) {
      nrm.resize((size_t)g.n * 4);
      CK(cudaMemcpyAsync(nrm.data(), g.d_norm45, nrm.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         c->stream), "copy norms");
      CK(cudaStreamSynchronize(c->stream), "step norms");
      for (int m = 0; m < g.n; ++m)
        for (int f = 0; f < 2; ++f) {
          const double u = nrm[(size_t)m * 4 + 2 + f], e = nrm[(size_t)m * 4 + f];
          if (u > 0.0) err = std::max(err, std::sqrt(e / u) * g.nx);
          else if (!(e >= 0.0)) err = NAN;
        }
    }
    if (!std::isfinite(err)) return fail(c, SBI_ENONFINITE, "the step error is not finite");
    if (err <= tol) {
      rc = launch_graph(c, gb);
      if (rc) return rc;
      ++acc;
      t = last ? t_end : t + hh;
      h = last ? std::max(h, next_step_size(hh, err, tol)) : next_step_size(hh, err, tol);
    } else {
      ++rej;
      h = next_step_size(hh, err, tol);
    }
    if (h < 1e-12 * std::fabs(span) || acc + rej > 10000000) {
      c->t_host = t;
      return fail(c, SBI_ENOTCONVERGED, "step size underflow at t = %.17g (h = %g)", t, h);
    }
  }
  c->t_host = t;
  *h_inout = h;
  if (accepted) *accepted = acc;
  if (rejected) *rejected = rej;
  if (c->opt.check_finite) return check_flags(c, "step");
  return SBI_OK;
}

int sbi_invariants(sbi_ctx* c, int member, double* mass, double* energy) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!mass || !energy) return fail(c, SBI_EINVAL, "mass and energy must not be NULL");
  const int gi = c->where[member].first;
  Group& g = c->groups[gi];
  rc = run_diag(c, gi, false);
  if (rc) return rc;
  const long long np = (long long)g.phys_elems();
  const size_t off = (size_t)c->where[member].second * np;
  const int chunk = 8192;
  const int nchunks = (int)((np + chunk - 1) / chunk);
  if ((size_t)nchunks * 2 > c->partial_cap) {
    void* p = dalloc(c, (size_t)nchunks * 2 * 8);
    if (!p) return fail(c, SBI_ENOMEM, "device allocation failed");
    c->d_partials = (double*)p;
    c->partial_cap = (size_t)nchunks * 2;
  }
  if (c->fp64)
    k_invariant_partials<double, false><<<nchunks, 256, 0, c->stream>>>(g.eta0 + off, g.phi0 + off, (const double*)g.Vphys + off, np, c->gravity, chunk, c->d_partials);
  else if (c->state_ds)
    k_invariant_partials<float, true><<<nchunks, 256, 0, c->stream>>>(g.eta0 + off, g.phi0 + off, (const float*)g.Vphys + off, np, c->gravity, chunk, c->d_partials);
  else
    k_invariant_partials<float, false><<<nchunks, 256, 0, c->stream>>>(g.eta0 + off, g.phi0 + off, (const float*)g.Vphys + off, np, c->gravity, chunk, c->d_partials);
  CK(cudaGetLastError(), "invariants");
  std::vector<double> part((size_t)nchunks * 2);
  CK(cudaMemcpyAsync(part.data(), c->d_partials, part.size() * 8, cudaMemcpyDeviceToHost, c->stream), "copy partials");
  CK(cudaStreamSynchronize(c->stream), "invariants");
  double m = 0.0, e = 0.0;
  for (int q = 0; q < nchunks; ++q) { m += part[2 * q]; e += part[2 * q + 1]; }
  const double dA = (g.Lx / g.nx) * (g.Ly / g.ny);
  *mass = m * dA;
  *energy = e * dA;
  return SBI_OK;
}

int ensure_time(sbi_ctx* c) {
  if (!c->d_time) {
    c->d_time = (double*)dalloc(c, sizeof(double));
    if (!c->d_time) return fail(c, SBI_ENOMEM, "device allocation failed");
  }
  CK(cudaStreamSynchronize(c->stream), "sync");
  CK(cudaMemcpy(c->d_time, &c->t_host, sizeof(double), cudaMemcpyHostToDevice), "copy time");
  return SBI_OK;
}

int sbi_set_time(sbi_ctx* c, double t) {
  if (!c) return SBI_EINVAL;
  if (!std::isfinite(t)) return fail(c, SBI_EINVAL, "t must be finite");
  c->t_host = t;
  return ensure_time(c);
}

int sbi_get_time(const sbi_ctx* c, double* t) {
  if (!c || !t) return SBI_EINVAL;
  *t = c->t_host;
  return SBI_OK;
}

int sbi_set_wavemaker(sbi_ctx* c, int ncomp, const double* amp, const double* omega,
                      const double* phase, double x0) {
  if (!c) return SBI_EINVAL;
  if (ncomp < 0 || ncomp > 256) return fail(c, SBI_EINVAL, "ncomp must be in 0..256");
  if (ncomp > 0 && c->opt.integrator == SBI_IF_RK45)
    return fail(c, SBI_EINVAL, "the wavemaker is not combined with integrator = SBI_IF_RK45");
  if (ncomp > 0 && (!amp || !omega || !phase)) return fail(c, SBI_EINVAL, "amp, omega and phase must not be NULL");
  if (!std::isfinite(x0)) return fail(c, SBI_EINVAL, "x0 must be finite");
  for (int j = 0; j < ncomp; ++j)
    if (!std::isfinite(amp[j]) || !(omega[j] > 0.0) || !std::isfinite(omega[j]) || !std::isfinite(phase[j]))
      return fail(c, SBI_EINVAL, "component %d: amp and phase must be finite, omega finite and > 0", j);
  CK(cudaStreamSynchronize(c->stream), "sync");
  CK(cudaStreamSynchronize(c->cap), "sync");
  free_graphs(c);   // the step's passes change
  c->wm_n = 0;
  if (ncomp == 0) return SBI_OK;
  int rc = ensure_time(c);
  if (rc) return rc;
  if (ncomp > c->wm_params_cap) {
    c->wm_params = (double*)dalloc(c, 2 * (size_t)ncomp * sizeof(double));
    if (!c->wm_params) return fail(c, SBI_ENOMEM, "device allocation failed");
    c->wm_params_cap = ncomp;
  }
  std::vector<double> par(2 * (size_t)ncomp);
  for (int j = 0; j < ncomp; ++j) {
    par[j] = omega[j];
    par[ncomp + j] = phase[j];
  }
  CK(cudaMemcpy(c->wm_params, par.data(), par.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
  const double bell = std::sqrt(std::exp(1.0) / (2.0 * M_PI));
  for (auto& g : c->groups) {
    if (ncomp > g.wm_cap) {
      g.wm_prof = (double*)dalloc(c, (size_t)ncomp * g.nx * sizeof(double));
      if (!g.wm_prof) return fail(c, SBI_ENOMEM, "device allocation failed");
      g.wm_cap = ncomp;
    }
    if (!g.wm_pg) {
      g.wm_pg = dalloc(c, (size_t)g.nx * c->real_size);
      if (!g.wm_pg) return fail(c, SBI_ENOMEM, "device allocation failed");
    }
    // bells g a_j sqrt(e/2pi) [1 + 2 k_j h0 / sinh(2 k_j h0)] exp(-(k_j d)^2 / 2),
    // omega_j^2 = g k_j tanh(k_j h0), d the periodic distance from x0
    std::vector<double> prof((size_t)ncomp * g.nx);
    for (int j = 0; j < ncomp; ++j) {
      const double w2 = omega[j] * omega[j];
      double k = w2 / c->gravity, shoal = 1.0;
      if (std::isfinite(g.h0)) {
        for (int it = 0; it < 100; ++it) {
          const double t = std::tanh(k * g.h0);
          const double dk = (c->gravity * k * t - w2) / (c->gravity * (t + k * g.h0 * (1.0 - t * t)));
          k -= dk;
          if (std::fabs(dk) <= 1e-15 * k) break;
        }
        shoal = 1.0 + 2.0 * k * g.h0 / std::sinh(2.0 * k * g.h0);
      }
      const double A = c->gravity * amp[j] * bell * shoal;
      for (int x = 0; x < g.nx; ++x) {
        const double xx = x * (g.Lx / g.nx);
        double d = std::fmod(xx - x0 + 0.5 * g.Lx, g.Lx);
        if (d < 0.0) d += g.Lx;
        d -= 0.5 * g.Lx;
        prof[(size_t)j * g.nx + x] = A * std::exp(-0.5 * (k * d) * (k * d));
      }
    }
    CK(cudaMemcpy(g.wm_prof, prof.data(), prof.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
  }
  c->wm_n = ncomp;
  return SBI_OK;
}

int sbi_orders_used(sbi_ctx* c, int member, int* orders) {
  int rc = check_member(c, member);
  if (rc) return rc;
  if (!orders) return fail(c, SBI_EINVAL, "orders is NULL");
  Group& g = c->groups[c->where[member].first];
  if (g.d_orders) {
    CK(cudaMemcpyAsync(orders, g.d_orders + c->where[member].second, sizeof(int),
                       cudaMemcpyDeviceToHost, c->stream), "orders");
    CK(cudaStreamSynchronize(c->stream), "orders");
  } else {
    *orders = c->opt.order;
  }
  return SBI_OK;
}

int sbi_profile_enable(sbi_ctx* c, int on) {
  if (!c) return SBI_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_graphs(c);
  c->prof = on != 0;
  c->prof_ms.assign(FAM_COUNT, 0.0);
  c->prof_launches.assign(FAM_COUNT, 0);
  return SBI_OK;
}

int sbi_profile_read(sbi_ctx* c, int cap, const char** names, long long* launches, double* total_ms,
                     int* count) {
  if (!c || !count) return SBI_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "profile sync");
  *count = FAM_COUNT;
  for (int i = 0; i < FAM_COUNT && i < cap; ++i) {
    if (names) names[i] = kFamilyNames[i];
    if (launches) launches[i] = i < (int)c->prof_launches.size() ? c->prof_launches[i] : 0;
    if (total_ms) total_ms[i] = i < (int)c->prof_ms.size() ? c->prof_ms[i] : 0.0;
  }
  return SBI_OK;
}

int sbi_step_bytes(const sbi_ctx* cc, int family, double* bytes) {
  sbi_ctx* c = const_cast<sbi_ctx*>(cc);
  if (!c || !bytes) return SBI_EINVAL;
  bool oom = false;
  std::vector<Pass> ps = plan_step(c, 1.0, &oom);
  if (oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  double b = 0.0;
  for (auto& p : ps)
    if (family < 0 || family_of(p) == family) b += p.bytes;
  *bytes = b;
  return SBI_OK;
}

int sbi_step_transforms(const sbi_ctx* cc, int family, double* point_transforms) {
  sbi_ctx* c = const_cast<sbi_ctx*>(cc);
  if (!c || !point_transforms) return SBI_EINVAL;
  bool oom = false;
  std::vector<Pass> ps = plan_step(c, 1.0, &oom);
  if (oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  double x = 0.0;
  for (auto& p : ps)
    if (family < 0 || family_of(p) == family) x += p.xforms;
  *point_transforms = x;
  return SBI_OK;
}

int sbi_step_launches(const sbi_ctx* cc, int* launches) {
  sbi_ctx* c = const_cast<sbi_ctx*>(cc);
  if (!c || !launches) return SBI_EINVAL;
  bool oom = false;
  std::vector<Pass> ps = plan_step(c, 1.0, &oom);
  if (oom) return fail(c, SBI_ENOMEM, "device allocation failed");
  *launches = (int)ps.size() + (c->wm_n > 0 ? 1 : 0);  // + the time advance
  return SBI_OK;
}

int sbi_autotune_report(const sbi_ctx* cc, char* buf, size_t cap, size_t* needed) {
  if (!cc || !needed || (cap > 0 && !buf)) return SBI_EINVAL;
  std::string out;
  for (const auto& key : cc->tune_order) {
    const auto& t = cc->tuned.at(key);
    char line[96];
    const bool row = key.rfind("row", 0) == 0;
    // column choices: "s" marks the staged form (inputs by bulk copies)
    snprintf(line, sizeof(line), ": %s %d%s/%d%s %.4f ms\n", row ? "rpc" : "cpb",
             row ? t.choice : t.choice % kStagedTag, (!row && t.choice >= kStagedTag) ? "s" : "",
             row ? t.deflt : t.deflt % kStagedTag, (!row && t.deflt >= kStagedTag) ? "s" : "", t.ms);
    out += key + line;
  }
  *needed = out.size();
  if (cap > 0) {
    const size_t n = out.size() < cap - 1 ? out.size() : cap - 1;
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return SBI_OK;
}

int sbi_test_stall_staged_copies(sbi_ctx* c, int on) {
  if (!c) return SBI_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "sync");
  free_graphs(c);   // the captured passes carry the old setting
  c->stall_tx = on ? 16 : 0;
  return SBI_OK;
}

int sbi_schedule_report(const sbi_ctx* cc, char* buf, size_t cap, size_t* needed) {
  if (!cc || !needed || (cap > 0 && !buf)) return SBI_EINVAL;
  const std::string& out = cc->sched_report;
  *needed = out.size();
  if (cap > 0) {
    const size_t n = out.size() < cap - 1 ? out.size() : cap - 1;
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return SBI_OK;
}

const char* sbi_last_error(const sbi_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void sbi_destroy(sbi_ctx* c) {
  if (!c) return;
  if (c->cap) cudaStreamSynchronize(c->cap);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto s2 : c->pstreams) cudaStreamSynchronize(s2);
  free_graphs(c);
  for (void* p : c->allocs) {
    if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_user);
    else cudaFree(p);
  }
  c->allocs.clear();
  for (auto s2 : c->gstreams) cudaStreamDestroy(s2);
  for (auto e2 : c->gevents) cudaEventDestroy(e2);
  for (auto s2 : c->pstreams) cudaStreamDestroy(s2);
  for (auto e2 : c->pevents) cudaEventDestroy(e2);
  for (auto e2 : c->tune_ev)
    if (e2) cudaEventDestroy(e2);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

}  // extern "C"
