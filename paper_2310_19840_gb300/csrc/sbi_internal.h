// sbi_internal.h - pass descriptors shared by the host planner and the kernels.
//
// One right-hand-side evaluation of the ESBI scheme is a chain of "row" and
// "column" passes over each member's fields.  Between passes a field lives in
// one of three layouts:
//   physical  ny x nx reals (x fastest);
//   mixed     W x ny complex, stored [kx][y]: FFT along x only, keeping the
//             W = ceil(alpha nx/2) non-negative x-modes that survive the dealias
//             mask (the Nyquist and all higher x-modes are zero by
//             construction), y physical, each kx column contiguous;
//   (spectral values exist only inside a column pass).
// A row pass turns mixed rows into physical ones (inverse real FFT along x),
// forms pointwise products, and turns them back into mixed rows (forward real
// FFT).  A column pass transforms mixed columns along y, applies per-mode
// multipliers k^p D(k) (i kx)^gx (i ky)^gy with D in {1, tanh(k h0),
// sech(k h0), Lambda(k)} and sums them into accumulators, masks, and
// transforms the outputs back along y.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace sbi {

constexpr int kMaxRowOps = 48;
constexpr int kMaxRowBufs = 40;
constexpr int kMaxColTerms = 48;
constexpr int kMaxColOuts = 12;
constexpr int kMaxColBufs = 32;
constexpr int kMaxColAcc = 2;
// threads of an RK stage block: rows per block = max(1, kRkThreads / threads per row)
constexpr int kRkThreads = 256;
constexpr int kMaxSlots = 5;
constexpr uint8_t kNone = 255;

enum RowOpKind : uint8_t {
  ROP_C2R = 0,   // slot <- c2r(sum of mixed bufs [a, a+b)); optional physical copy to dst
  ROP_PROD = 1,  // mixed dst <- r2c(coef * eta^a * delta^b * w^(c&1) * slot)  (slot kNone: 1);
                 // c & 2: running product, the slot itself becomes eta^a delta^b slot
  ROP_N2 = 2,    // mixed dst <- r2c(dynamic-condition right-hand side) from slots
                 // slot..slot+4 = V, eta_x, eta_y, phi_x, phi_y (2-D) or
                 // V, eta_x, phi_x (1-D); coef = gravity
  ROP_WDOT = 3,  // physical dst <- w-free Eulerian vertical velocity
                 // (V + grad eta.grad phi)/(1+|grad eta|^2) from the same slots
  ROP_VFW = 4,   // mixed dst <- r2c(W (1 + |grad eta|^2) - grad eta.grad phi), the
                 // kinematic V from the Eulerian W in the V slot (HOS diagnostic)
};

struct RowOp {
  uint8_t kind;
  uint8_t slot;
  uint8_t a;
  uint8_t b;
  uint8_t c;
  uint8_t dst;
  uint16_t pad_;
  uint32_t pad2_;
  double coef;    // PROD: scalar coefficient; N2: gravity
};

struct BufRef {
  void* ptr;
  long long stride;   // elements (reals for physical, complex for mixed) between members
};

struct RowParams {
  int rpc;              // rows per block (runtime, <= the kernel's maximum)
  int nops;
  int row_begin;        // first row of this launch (a member range starts at member * ny)
  int rows_total;       // end of the launch's rows: members * ny for the whole group
  int ny;
  int W;
  int nslots;
  int fbs, sws;         // row strides of the FFT scratch and staging rows (set by the launcher)
  int member0;          // first member of this launch within the group (for convergence flags)
  const int* active;    // per-member flag (nullptr: all active); inactive members skip the pass
  BufRef eta, delta, wgt;        // physical fields (ptr may be null)
  const void* pg;       // surface pressure / rho along x (nx reals, the same for
                        // every row), subtracted by ROP_N2; nullptr: none
  BufRef buf[kMaxRowBufs];
  RowOp ops[kMaxRowOps];
  const void* tw;
};

// One multiplier of a column pass: c k^p D(k) (i kx)^gx (i ky)^gy, times the
// dealias mask M (mask = 1) or (M D - 1) without D elsewhere (mask = 2).  The
// real factor is tabulated per mode once per context (tab, layout [kx][ny]);
// the kernels apply tab and the phase i^(gx+gy).
struct ColTerm {
  const void* tab; // per-mode real factor in the working precision
  uint8_t in;     // input buffer (local index); for outputs: destination buffer
  uint8_t acc;    // accumulator index
  uint8_t gx, gy; // powers of (i kx), (i ky)
  int8_t kpow;    // power of |k| (negative powers vanish at k = 0)
  uint8_t depth;  // 0: 1, 1: tanh(k h0), 2: sech(k h0), 3: Lambda(k) = exp(-(k/kf)^beta2);
                  // entries of the linear propagator e^{A tau}, w^2 = g k tanh(k h0):
                  // 4: cos(w tau) - 1, 5: (k tanh(k h0) / w) sin(w tau), 6: (g / w) sin(w tau)
                  // (g tau at k = 0), 7: cos(w tau); factors of the implicit form of
                  // Appendix A, e_h = e^{-2 k h0}: 8: 1 + e_h (C_h^-1), 9: 1 - e_h
                  // (D_h^-1), 10: e_h, 11: 1 / (1 + e_h) (C_h), 12: sqrt(e_h),
                  // 13: 1 / (1 - e_h) (D_h; 0 at k = 0)
  uint8_t mask;   // 0: none, 1: dealias mask, 2: (mask * D - 1) projection correction
  uint8_t pad_;
  double c;
  double tau;     // time of the propagator entries (depth 4..7) [s]
};

struct ColParams {
  int nin, nterms, nouts, nacc;
  int cpb;                  // columns per block (0: the size's default; see col_cpb_ok)
  int W, ny, nx;
  int col_begin;            // first column of this launch (a member range starts at member * W)
  int cols_total;           // end of the launch's columns: members * W for the whole group
  int member0;
  const int* active;
  double two_pi_over_Lx, two_pi_over_Ly, h0;
  int kx_keep, ky_keep;     // keep m < kx_keep and |n| < ky_keep
  double filt_kf, filt_beta2;
  double* norm_out;         // optional per-member FP64 partial norms of accumulator 0 (nullptr: off)
  int staged;               // 1: inputs staged in shared memory by bulk copies (sizes >= 32)
  int* err_flag;            // set to 1 when a bounded wait of the staged form gave up
  int npass;                // mixed buffers added unchanged to output 0 after its inverse FFT
  BufRef pass[8];
  int term_begin[kMaxColBufs + 1];   // terms sorted by input
  ColTerm terms[kMaxColTerms];
  ColTerm outs[kMaxColOuts];
  BufRef buf[kMaxColBufs];
  const void* tw;
  int stall_tx;             // test hook: bytes a staged copy's barrier expects beyond the copy
                            // (0; > 0 makes every wait run out, to test the timeout path)
};

// Parameters of one multiplier table (see ColTerm).
struct TableSpec {
  int W, ny, kx_keep, ky_keep;
  double two_pi_over_Lx, two_pi_over_Ly, h0, filt_kf, filt_beta2, c;
  double tau, gravity;  // propagator entries (depth 4..7)
  int kpow, depth, gx, gy, mask;
};

// RK_ENTRY: working copies of the state; RK_STAGE: a classical RK4 stage;
// RK_CORRECT: add two mixed corrections to the state, then working copies;
// RK_OFFSET: working copies of the state plus two mixed offsets, the state
// itself unchanged (the intermediate stages of the integrating-factor scheme)
enum RkMode : int { RK_ENTRY = 0, RK_STAGE = 1, RK_CORRECT = 2, RK_OFFSET = 3 };

// A step-size scalar of the RK stage update in both representations: the
// double, and its double-single split (hi = nearest float, lo = nearest float
// of the rest), formed on the host so that the state update never rounds the
// step to a float.
struct RkScalar {
  double d;
  float hi, lo;
};

struct RkParams {
  int rpc;              // rows per block
  int fbs;              // row stride of the scratch rows (set by the launcher)
  const int* active;    // per-member flag (nullptr: all members)
  int mode;             // RkMode
  int stage;            // 1..4 for RK_STAGE
  int tail;             // 1: write the next stage's working copies (eta_w, mixed eta^, phi^)
  int row_begin;        // first row of this launch (a member range starts at member * ny)
  int rows_total, ny, W;  // rows_total: end of the launch's rows
  double dt;
  int state64;          // FP32 path only: the state and sums are FP64 (else double-single)
  RkScalar dt6, cdt;    // RK_STAGE: dt/6 (stage 4 update) and the stage's offset c dt
  BufRef eta0, phi0;    // master state (FP64, or double-single pairs)
  BufRef acc_eta, acc_phi;      // RK4 sums k1 + 2 k2 + 2 k3 + k4 (state format)
  BufRef V;             // physical V of this stage (T)
  BufRef phit;          // mixed phi~_t of this stage (T complex) / RK_CORRECT, RK_OFFSET: eta correction
  BufRef corr_phi;      // RK_CORRECT, RK_OFFSET: phi correction (mixed)
  BufRef eta_w;         // physical working eta (T)
  BufRef eta_hat, phi_hat;      // mixed working spectra (T complex)
  int* nonfinite;       // set to 1 when the new state holds NaN/Inf
  const void* tw;
};

// Launchers (one instantiation per real type and size, selected at run time).
// prepare_kernels sets the dynamic shared-memory limits of every kernel a
// grid of nx x ny uses; it must run once (outside stream capture) before the
// first launch.  Unsupported sizes return cudaErrorInvalidValue.
template <typename T> cudaError_t prepare_row_kernels(int nx);
template <typename T> cudaError_t prepare_col_kernels(int ny);
struct TableSpec;
template <typename T> cudaError_t launch_coef_table(void* out, const TableSpec& s, cudaStream_t st);
template <typename T> cudaError_t launch_row(int nx, const RowParams& p, cudaStream_t st);
template <typename T> cudaError_t launch_col(int ny, const ColParams& p, cudaStream_t st);
template <typename T> cudaError_t launch_rk(int nx, const RkParams& p, cudaStream_t st);
// Convert n state values between host-visible doubles and the state storage
// of the working precision (double, or hi/lo float pairs for FP32).
template <typename T> cudaError_t state_convert(const void* src, void* dst, long long n, bool to_double,
                                                cudaStream_t st);
// rows per block for a row pass with nslots physical slots (0: does not fit)
template <typename T> int row_rpc(int nx, int W, int nslots);
// launch geometry of a size: threads per row of a row pass; default columns
// per block and threads per column of a column pass (0 for an unknown size)
template <typename T> int row_tpr(int nx);
template <typename T> int col_geometry(int ny, int* tpc);
// whether columns of ny points can take the staged (bulk-copy) form
template <typename T> bool col_stageable(int ny);

}  // namespace sbi
