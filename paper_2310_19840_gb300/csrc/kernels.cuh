// kernels.cuh - row, column and RK4 passes of the ESBI step (templates).
//
// Layouts (see sbi_internal.h): physical fields are [member][y][x]; mixed
// fields (x-spectral, y-physical, only the W kept x-modes) are stored
// transposed, [member][kx][y], so that a column pass reads each column as one
// contiguous run.  A row pass handles `rpc` rows per block, one group of TPR
// threads per row; its FFTs are warp-synchronous when TPR <= 32.  Mixed rows
// are moved between global memory and per-row shared-memory buffers by the
// whole block (rpc consecutive y per kx, i.e. coalesced runs of rpc complex).
//
// Included by the per-type instantiation units only.
#pragma once

#include <math.h>

#include "fft.cuh"
#include "sbi_internal.h"

namespace sbi {

// ===========================================================================
// Row passes
// ===========================================================================
template <int NX>
struct RowCfg {
  static constexpr int n = NX / 2;                       // packed complex length
  static constexpr int R = (n >= 128) ? 16 : cmin(8, n); // elements per thread
  static constexpr int TPR = n / R;                      // threads per row
  static constexpr bool WARP = TPR <= 32;
  static constexpr int RPC_MAX = cmin(256, WARP ? cmax(16, 256 / TPR) : cmax(1, 512 / TPR));
  static constexpr int MAX_THREADS = TPR * RPC_MAX;
  static constexpr int FBUF = padded_len(n);
};

// shared memory of a row block: per row the FFT scratch (which also stages
// the incoming mixed row), the row of eta, and the physical slots
template <typename T, int NX>
__host__ __device__ constexpr size_t row_smem(int rpc, int W, int nslots) {
  using C = RowCfg<NX>;
  (void)W;
  return sizeof(cx<T>) * (size_t)rpc * ((size_t)C::FBUF + (size_t)(1 + nslots) * C::n);
}

template <int NX>
__device__ __forceinline__ void row_group_sync() {
  if constexpr (RowCfg<NX>::WARP) __syncwarp();
  else __syncthreads();
}

// physical row viewed as n complex pairs (x[2m], x[2m+1])
template <typename T>
__device__ __forceinline__ const cx<T>* phys_row(const BufRef& b, int member, int y, int NX) {
  return reinterpret_cast<const cx<T>*>(reinterpret_cast<const T*>(b.ptr) +
                                        (long long)member * b.stride + (long long)y * NX);
}
template <typename T>
__device__ __forceinline__ cx<T>* phys_row_w(const BufRef& b, int member, int y, int NX) {
  return reinterpret_cast<cx<T>*>(reinterpret_cast<T*>(b.ptr) + (long long)member * b.stride +
                                  (long long)y * NX);
}
// element (kx, y) of a member's mixed field
__device__ __forceinline__ long long mixed_index(long long stride, int member, int kx, int y, int ny) {
  return (long long)member * stride + (long long)kx * ny + y;
}

// Geometry of the block-cooperative mixed I/O.  blockDim = rpc * TPR, rpc a
// power of two, so thread t always serves row rl = t % rpc and the modes
// k = t / rpc + i * TPR: the row's member, y and flags are computed once.
struct RowIO {
  int rl, k0, kstep, W, ny;
  bool ok;                 // row exists and its member is active
  long long base;          // member * stride + y of this thread's row (stride added per buffer)
  int member, y;
  __device__ __forceinline__ RowIO(int row0, int rpc, int rows_total, int ny_, int W_,
                                   const int* active, int member0) {
    rl = threadIdx.x & (rpc - 1);
    k0 = threadIdx.x / rpc;
    kstep = blockDim.x / rpc;
    W = W_;
    ny = ny_;
    const int row = row0 + rl;
    ok = row < rows_total;
    member = ok ? row / ny : 0;
    y = ok ? row - member * ny : 0;
    if (ok && active) ok = active[member0 + member] != 0;
    base = y;
  }
  __device__ __forceinline__ long long at(const BufRef& b, int k) const {
    return (long long)member * b.stride + (long long)k * ny + base;
  }
};

// Block-cooperative load of the mixed rows (sum of nb buffers) into the
// per-row scratch, stg[rl * FBUF + k], k < W.
template <typename T>
__device__ __forceinline__ void stage_mixed(cx<T>* stg_all, int fbuf, const BufRef* bufs, int nb,
                                            const RowIO& io) {
  using V = cx<T>;
  V* stg = stg_all + io.rl * fbuf;
  for (int k = io.k0; k < io.W; k += io.kstep) {
    V a = mk<V>(T(0), T(0));
    if (io.ok) {
      for (int q = 0; q < nb; ++q) a = cadd(a, reinterpret_cast<const V*>(bufs[q].ptr)[io.at(bufs[q], k)]);
    }
    stg[k] = a;
  }
}

// Packed inverse real FFT, input side, from the staged row: Z[k] = E + i O,
// E = X[k] + X*[n-k], O = (X[k] - X*[n-k]) e^{+2 pi i k / NX}, k = j + r TPR;
// X[k] = 0 for k >= W, and the Nyquist mode X[n] = 0.  The unnormalised
// inverse of Z gives NX * x packed as z[m] = x[2m] + i x[2m+1].
template <typename T, int NX>
__device__ __forceinline__ void c2r_input(cx<T> (&x)[RowCfg<NX>::R], const cx<T>* stg, int W, int j,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    const int k = j + r * C::TPR;
    const int kk = C::n - k;
    const V a = (k < W) ? stg[k] : mk<V>(T(0), T(0));
    const V b = (k > 0 && kk < W) ? stg[kk] : mk<V>(T(0), T(0));
    const V bc = cconj(b);
    const V E = cadd(a, bc);
    const V O = cmul(csub(a, bc), cconj(__ldg(tw + tw_off(NX) + k)));
    x[r] = cadd(E, rot<1>(O));
  }
}

// Packed forward real FFT, output side, block-cooperative: each row's
// natural-order Z is in fb[rl]; the kept modes
// X[k] = 1/2 (Z[k] + Z*[n-k]) - i/2 e^{-2 pi i k / NX} (Z[k] - Z*[n-k]), k < W,
// are written to the transposed mixed field dst.
template <typename T, int NX>
__device__ __forceinline__ void r2c_store(const cx<T>* fb_all, const BufRef& dst, const RowIO& io,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  if (!io.ok) return;
  V* out = reinterpret_cast<V*>(dst.ptr);
  const V* fb = fb_all + io.rl * C::FBUF;
  for (int k = io.k0; k < io.W; k += io.kstep) {
    const V zk = fb[pad(k)];
    const V zc = cconj(fb[pad((C::n - k) & (C::n - 1))]);
    const V s = cadd(zk, zc);
    const V d = cmul(csub(zk, zc), __ldg(tw + tw_off(NX) + k));
    out[io.at(dst, k)] = cscale(csub(s, rot<1>(d)), T(0.5));
  }
}

template <typename T>
__device__ __forceinline__ T ipow(T v, int p) {
  T r = T(1);
  for (int i = 0; i < p; ++i) r *= v;
  return r;
}

template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<NX>::MAX_THREADS)
k_row(const __grid_constant__ RowParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = p.rpc;
  V* fb_all = reinterpret_cast<V*>(smem_raw);      // FFT scratch, also staging
  V* eta_all = fb_all + rpc * C::FBUF;             // rows of eta (pairs)
  V* slot_base = eta_all + rpc * n;                // physical slots
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  V* fb = fb_all + rloc * C::FBUF;
  V* eta = eta_all + rloc * n;
  const int row0 = (int)blockIdx.x * rpc;
  const RowIO io(row0, rpc, p.rows_total, p.ny, p.W, p.active, p.member0);
  const int row = row0 + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row - member * p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);

  if (p.eta.ptr) {
    const V* er = act ? phys_row<T>(p.eta, member, y, NX) : nullptr;
#pragma unroll
    for (int r = 0; r < R; ++r) eta[j + r * TPR] = er ? er[j + r * TPR] : mk<V>(T(0), T(0));
  }

  for (int o = 0; o < p.nops; ++o) {
    const RowOp op = p.ops[o];
    V x[R];
    if (op.kind == ROP_C2R) {
      __syncthreads();  // scratch free (previous cooperative store done)
      stage_mixed<T>(fb_all, C::FBUF, p.buf + op.a, op.b, io);
      __syncthreads();
      c2r_input<T, NX>(x, fb, p.W, j, tw);
      row_group_sync<NX>();  // the staged row is read before the FFT overwrites it
      fft_block<n, R, +1>(x, fb, j, tw);
      V* slot = slot_base + (op.slot * rpc + rloc) * n;
      V* out = (act && op.dst != kNone) ? phys_row_w<T>(p.buf[op.dst], member, y, NX) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V z = fb[pad(m)];
        slot[m] = z;
        if (out) out[m] = z;
      }
      continue;
    }
    if (op.kind == ROP_PROD) {
      const V* slot = op.slot == kNone ? nullptr : slot_base + (op.slot * rpc + rloc) * n;
      const T cf = T(op.coef);
      const V* drow = (act && op.b > 0 && p.delta.ptr) ? phys_row<T>(p.delta, member, y, NX) : nullptr;
      const V* wrow = (act && op.c > 0 && p.wgt.ptr) ? phys_row<T>(p.wgt, member, y, NX) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V v = slot ? slot[m] : mk<V>(T(1), T(1));
        const V e = eta[m];
        T f0 = cf * ipow(e.x, op.a), f1 = cf * ipow(e.y, op.a);
        if (drow) {
          const V d = drow[m];
          f0 *= ipow(d.x, op.b);
          f1 *= ipow(d.y, op.b);
        }
        if (wrow) {
          const V w = wrow[m];
          f0 *= w.x;
          f1 *= w.y;
        }
        x[r] = mk<V>(f0 * v.x, f1 * v.y);
      }
    } else {
      // ROP_N2 / ROP_WDOT: slots V, eta_x, [eta_y,] phi_x, [phi_y]
      const bool two_d = op.a == 2;
      const V* sV = slot_base + ((op.slot + 0) * rpc + rloc) * n;
      const V* sEx = slot_base + ((op.slot + 1) * rpc + rloc) * n;
      const V* sEy = two_d ? slot_base + ((op.slot + 2) * rpc + rloc) * n : nullptr;
      const V* sPx = slot_base + ((op.slot + (two_d ? 3 : 2)) * rpc + rloc) * n;
      const V* sPy = two_d ? slot_base + ((op.slot + 4) * rpc + rloc) * n : nullptr;
      const T g = T(op.coef);
      V* wout = (op.kind == ROP_WDOT && act) ? phys_row_w<T>(p.buf[op.dst], member, y, NX) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V vv = sV[m], ex = sEx[m], px = sPx[m];
        const V ey = two_d ? sEy[m] : mk<V>(T(0), T(0));
        const V py = two_d ? sPy[m] : mk<V>(T(0), T(0));
        const V e = eta[m];
        T res[2];
        const T vc[2] = {vv.x, vv.y}, exc[2] = {ex.x, ex.y}, eyc[2] = {ey.x, ey.y};
        const T pxc[2] = {px.x, px.y}, pyc[2] = {py.x, py.y}, ec[2] = {e.x, e.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const T dot = exc[h] * pxc[h] + eyc[h] * pyc[h];
          const T ge2 = exc[h] * exc[h] + eyc[h] * eyc[h];
          const T gp2 = pxc[h] * pxc[h] + pyc[h] * pyc[h];
          const T num = vc[h] + dot;
          if (op.kind == ROP_N2)
            res[h] = -g * ec[h] + T(0.5) * (num * num / (T(1) + ge2) - gp2);
          else
            res[h] = num / (T(1) + ge2);
        }
        x[r] = mk<V>(res[0], res[1]);
        if (wout) wout[m] = x[r];
      }
      if (op.kind == ROP_WDOT) continue;
    }
    __syncthreads();  // scratch free (previous cooperative store done)
    fft_block<n, R, -1>(x, fb, j, tw);
    __syncthreads();  // every row's spectrum ready
    r2c_store<T, NX>(fb_all, p.buf[op.dst], io, tw);
  }
}

// ===========================================================================
// RK4 stage pass (row layout).  FP64 state and sums for every real type.
// ===========================================================================
template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<NX>::MAX_THREADS)
k_rk(const __grid_constant__ RkParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = p.rpc;
  V* fb_all = reinterpret_cast<V*>(smem_raw);
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  V* fb = fb_all + rloc * C::FBUF;
  const int row0 = (int)blockIdx.x * rpc;
  const RowIO io(row0, rpc, p.rows_total, p.ny, p.W, p.active, 0);
  const int row = row0 + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row - member * p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const long long off = (long long)y * NX;

  // new state in the working precision (the FFT inputs of the tail)
  V xe[R], xp[R];
  const double* E0 = reinterpret_cast<const double*>(p.eta0.ptr) + member * p.eta0.stride + off;
  const double* P0 = reinterpret_cast<const double*>(p.phi0.ptr) + member * p.phi0.stride + off;
  double* E0w = reinterpret_cast<double*>(p.eta0.ptr) + member * p.eta0.stride + off;
  double* P0w = reinterpret_cast<double*>(p.phi0.ptr) + member * p.phi0.stride + off;
  bool bad = false;

  if (p.mode == RK_ENTRY) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = j + r * TPR;
      const double2 e = act ? reinterpret_cast<const double2*>(E0)[m] : make_double2(0.0, 0.0);
      const double2 q = act ? reinterpret_cast<const double2*>(P0)[m] : make_double2(0.0, 0.0);
      xe[r] = mk<V>(T(e.x), T(e.y));
      xp[r] = mk<V>(T(q.x), T(q.y));
    }
  } else {
    V x[R];
    // first inverse: phi~_t (stage) or the eta correction
    stage_mixed<T>(fb_all, C::FBUF, &p.phit, 1, io);
    __syncthreads();
    c2r_input<T, NX>(x, fb, p.W, j, tw);
    row_group_sync<NX>();
    fft_block<n, R, +1>(x, fb, j, tw);
    if (p.mode == RK_CORRECT) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V c = fb[pad(m)];
        double2 e = act ? reinterpret_cast<const double2*>(E0)[m] : make_double2(0.0, 0.0);
        e.x += double(c.x);
        e.y += double(c.y);
        if (act) reinterpret_cast<double2*>(E0w)[m] = e;
        bad |= !isfinite(e.x) || !isfinite(e.y);
        xe[r] = mk<V>(T(e.x), T(e.y));
      }
      __syncthreads();
      stage_mixed<T>(fb_all, C::FBUF, &p.corr_phi, 1, io);
      __syncthreads();
      c2r_input<T, NX>(x, fb, p.W, j, tw);
      row_group_sync<NX>();
      fft_block<n, R, +1>(x, fb, j, tw);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V c = fb[pad(m)];
        double2 q = act ? reinterpret_cast<const double2*>(P0)[m] : make_double2(0.0, 0.0);
        q.x += double(c.x);
        q.y += double(c.y);
        if (act) reinterpret_cast<double2*>(P0w)[m] = q;
        bad |= !isfinite(q.x) || !isfinite(q.y);
        xp[r] = mk<V>(T(q.x), T(q.y));
      }
    } else {
      // classical RK4: sums b = (1/6, 1/3, 1/3, 1/6), next-stage offsets c = (1/2, 1/2, 1)
      const V* Vr = act ? phys_row<T>(p.V, member, y, NX) : nullptr;
      double2* AE = reinterpret_cast<double2*>(reinterpret_cast<double*>(p.acc_eta.ptr) + member * p.acc_eta.stride + off);
      double2* AP = reinterpret_cast<double2*>(reinterpret_cast<double*>(p.acc_phi.ptr) + member * p.acc_phi.stride + off);
      const double bw = (p.stage == 1 || p.stage == 4) ? (1.0 / 6.0) : (1.0 / 3.0);
      const double cn = (p.stage == 3) ? 1.0 : 0.5;
      const double dt = p.dt;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V ft = fb[pad(m)];
        double2 e = make_double2(0.0, 0.0), q = make_double2(0.0, 0.0);
        if (act) {
          const V vv = Vr[m];
          const double2 e0 = reinterpret_cast<const double2*>(E0)[m];
          const double2 q0 = reinterpret_cast<const double2*>(P0)[m];
          double2 ae = make_double2(bw * double(vv.x), bw * double(vv.y));
          double2 ap = make_double2(bw * double(ft.x), bw * double(ft.y));
          if (p.stage > 1) {
            const double2 a0 = AE[m], b0 = AP[m];
            ae.x += a0.x; ae.y += a0.y;
            ap.x += b0.x; ap.y += b0.y;
          }
          if (p.stage < 4) {
            AE[m] = ae;
            AP[m] = ap;
            e = make_double2(e0.x + cn * dt * double(vv.x), e0.y + cn * dt * double(vv.y));
            q = make_double2(q0.x + cn * dt * double(ft.x), q0.y + cn * dt * double(ft.y));
          } else {
            e = make_double2(e0.x + dt * ae.x, e0.y + dt * ae.y);
            q = make_double2(q0.x + dt * ap.x, q0.y + dt * ap.y);
            reinterpret_cast<double2*>(E0w)[m] = e;
            reinterpret_cast<double2*>(P0w)[m] = q;
            bad |= !isfinite(e.x) || !isfinite(e.y) || !isfinite(q.x) || !isfinite(q.y);
          }
        }
        xe[r] = mk<V>(T(e.x), T(e.y));
        xp[r] = mk<V>(T(q.x), T(q.y));
      }
    }
  }
  if (bad && p.nonfinite) *p.nonfinite = 1;

  if (!p.tail) return;
  // working copies of the next stage: physical eta, mixed eta^ and phi^
  V* ew = act ? phys_row_w<T>(p.eta_w, member, y, NX) : nullptr;
  if (ew) {
#pragma unroll
    for (int r = 0; r < R; ++r) ew[j + r * TPR] = xe[r];
  }
  __syncthreads();
  fft_block<n, R, -1>(xe, fb, j, tw);
  __syncthreads();
  r2c_store<T, NX>(fb_all, p.eta_hat, io, tw);
  __syncthreads();
  fft_block<n, R, -1>(xp, fb, j, tw);
  __syncthreads();
  r2c_store<T, NX>(fb_all, p.phi_hat, io, tw);
}

// ===========================================================================
// Column pass: CPB columns per block, TPC threads per column (one warp or less
// per column up to NY = 512), each column a contiguous run of NY complex.
// ===========================================================================
template <int NY>
struct ColCfg {
  static constexpr int RC = NY == 1 ? 1 : (NY <= 256 ? cmin(8, NY) : 16);
  static constexpr int TPC = NY / RC;
  static constexpr bool WARP = TPC <= 32;
  static constexpr int CPB = NY == 1 ? 256 : cmax(1, 256 / TPC);
  static constexpr int THREADS = TPC * CPB;
  static constexpr int CBUF = padded_len(NY);
};

// per column: FFT scratch and the (tanh, sech) factors of its modes
template <typename T, int NY>
__host__ __device__ constexpr size_t col_smem() {
  return sizeof(cx<T>) * (size_t)ColCfg<NY>::CPB * ((NY == 1 ? 0 : ColCfg<NY>::CBUF) + NY);
}

// c k^p D (i kx)^gx (i ky)^gy x  (negative powers of k vanish at k = 0).  The
// term is uniform across the block, so its fields select without divergence.
template <typename T>
__device__ __forceinline__ cx<T> apply_term(const ColTerm& t, cx<T> x, T k, T kxv, T kyv, T tk,
                                            T sk, T lam) {
  using V = cx<T>;
  const int ap = t.kpow < 0 ? -t.kpow : t.kpow;
  T kp = T(1);
  for (int i = 0; i < ap; ++i) kp *= k;
  if (t.kpow < 0) kp = (k > T(0)) ? T(1) / kp : T(0);
  T f = T(t.c) * kp;
  f *= (t.depth == 1) ? tk : ((t.depth == 2) ? sk : ((t.depth == 3) ? lam : T(1)));
  f *= (t.gx ? kxv : T(1)) * (t.gx == 2 ? kxv : T(1)) * (t.gy ? kyv : T(1)) * (t.gy == 2 ? kyv : T(1));
  const int q = (t.gx + t.gy) & 3;   // multiply by i^q
  const T re = x.x * f, im = x.y * f;
  T r2 = (q & 1) ? -im : re;
  T i2 = (q & 1) ? re : im;
  if (q & 2) {
    r2 = -r2;
    i2 = -i2;
  }
  return mk<V>(r2, i2);
}

// tanh(k h0) and sech(k h0) = 2 e^{-k h0} / (1 + e^{-2 k h0}); deep water for h0 = inf
template <typename T>
__device__ __forceinline__ void depth_factors(T k, T h0, bool deep, T& tk, T& sk) {
  if (!(k > T(0))) {
    tk = T(0);
    sk = T(1);
  } else if (deep) {
    tk = T(1);
    sk = T(0);
  } else {
    const T kh = k * h0;
    const T e = exp(-kh);
    tk = tanh(kh);
    sk = T(2) * e / (T(1) + e * e);
  }
}

template <typename T>
__device__ __forceinline__ T filter_factor(T k, T kf, T beta2) {
  return kf > T(0) ? exp(-pow(k / kf, beta2)) : T(1);
}

template <typename T, int NY, int NACC>
__global__ void __launch_bounds__(ColCfg<NY>::THREADS)
k_col(const __grid_constant__ ColParams p) {
  using V = cx<T>;
  using C = ColCfg<NY>;
  constexpr int RC = C::RC, TPC = C::TPC, CPB = C::CPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x / TPC, j = threadIdx.x % TPC;
  constexpr int SCR = NY == 1 ? 0 : C::CBUF;
  V* sc = reinterpret_cast<V*>(smem_raw) + c * SCR;
  V* dts = reinterpret_cast<V*>(smem_raw) + CPB * SCR + c * NY;   // (tanh, sech) per mode
  const int gc = blockIdx.x * CPB + c;
  const bool valid = gc < p.cols_total;
  const int member = valid ? gc / p.W : 0;
  const int kx = valid ? gc % p.W : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const bool deep = isinf(p.h0);
  const T h0 = deep ? T(0) : T(p.h0);
  const T kxv = T(kx) * T(p.two_pi_over_Lx);
  const T ky1 = T(p.two_pi_over_Ly);
  const long long col_off = (long long)kx * NY;

  // depth factors of the thread's modes n = j + r TPC (read back only by this thread)
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    const int ni = j + r * TPC;
    const int ns = (NY == 1) ? 0 : (ni < NY / 2 ? ni : ni - NY);
    const T kyv = T(ns) * ky1;
    T tk, sk;
    depth_factors<T>(sqrt(kxv * kxv + kyv * kyv), h0, deep, tk, sk);
    dts[ni] = mk<V>(tk, sk);
  }

  V acc[NACC][RC];
#pragma unroll
  for (int a = 0; a < NACC; ++a)
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[a][r] = mk<V>(T(0), T(0));
  for (int i = 0; i < p.nin; ++i) {
    V x[RC];
    const V* src = reinterpret_cast<const V*>(p.buf[i].ptr) + member * p.buf[i].stride + col_off;
#pragma unroll
    for (int r = 0; r < RC; ++r) x[r] = act ? src[j + r * TPC] : mk<V>(T(0), T(0));
    if constexpr (NY > 1) {
      group_sync<C::WARP>();  // scratch free
      fft_block<NY, RC, -1>(x, sc, j, tw);
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = sc[pad(j + r * TPC)];
    }
    for (int q = p.term_begin[i]; q < p.term_begin[i + 1]; ++q) {
      const ColTerm t = p.terms[q];
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const int ni = j + r * TPC;
        const int ns = (NY == 1) ? 0 : (ni < NY / 2 ? ni : ni - NY);
        const T kyv = T(ns) * ky1;
        const T kk = sqrt(kxv * kxv + kyv * kyv);
        const V ts = dts[ni];
        const V v = apply_term<T>(t, x[r], kk, kxv, kyv, ts.x, ts.y, T(1));
        if (NACC == 1 || t.acc == 0) acc[0][r] = cadd(acc[0][r], v);
        else acc[NACC - 1][r] = cadd(acc[NACC - 1][r], v);
      }
    }
  }
  for (int o = 0; o < p.nouts; ++o) {
    const ColTerm t = p.outs[o];
    V x[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      const int ni = j + r * TPC;
      const int ns = (NY == 1) ? 0 : (ni < NY / 2 ? ni : ni - NY);
      const T kyv = T(ns) * ky1;
      const T kk = sqrt(kxv * kxv + kyv * kyv);
      const bool keep = kx < p.kx_keep && (ns < 0 ? -ns : ns) < p.ky_keep;
      const T lam = (t.depth == 3) ? filter_factor<T>(kk, T(p.filt_kf), T(p.filt_beta2)) : T(1);
      const V a = (NACC == 1 || t.acc == 0) ? acc[0][r] : acc[NACC - 1][r];
      if (t.mask == 2) {
        // (M D - 1) a: projection correction, D = Lambda (depth 3) or 1
        ColTerm u = t;
        u.depth = 0;
        const T mfac = (keep ? lam : T(0)) - T(1);
        x[r] = cscale(apply_term<T>(u, a, kk, kxv, kyv, T(0), T(0), lam), mfac);
      } else {
        const V ts = dts[ni];
        x[r] = apply_term<T>(t, a, kk, kxv, kyv, ts.x, ts.y, lam);
        if (t.mask == 1 && !keep) x[r] = mk<V>(T(0), T(0));
      }
    }
    if constexpr (NY > 1) {
      group_sync<C::WARP>();
      fft_block<NY, RC, +1>(x, sc, j, tw);
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = sc[pad(j + r * TPC)];
    }
    if (act) {
      V* dst = reinterpret_cast<V*>(p.buf[t.in].ptr) + member * p.buf[t.in].stride + col_off;
#pragma unroll
      for (int r = 0; r < RC; ++r) dst[j + r * TPC] = x[r];
    }
  }
}

// ===========================================================================
// Launchers
// ===========================================================================
template <typename T, int NX>
cudaError_t prepare_nx() {
  const int maxb = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_row<T, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rk<T, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
}

template <typename T, int NY>
cudaError_t prepare_ny() {
  cudaError_t e = cudaFuncSetAttribute(k_col<T, NY, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)col_smem<T, NY>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_col<T, NY, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)col_smem<T, NY>());
}

template <typename T, int NX>
cudaError_t launch_row_n(const RowParams& p, cudaStream_t st) {
  using C = RowCfg<NX>;
  if (p.rpc < 1 || p.rpc > C::RPC_MAX) return cudaErrorInvalidValue;
  const int blocks = (p.rows_total + p.rpc - 1) / p.rpc;
  k_row<T, NX><<<blocks, C::TPR * p.rpc, row_smem<T, NX>(p.rpc, p.W, p.nslots), st>>>(p);
  return cudaGetLastError();
}

template <typename T, int NX>
cudaError_t launch_rk_n(const RkParams& p, cudaStream_t st) {
  using C = RowCfg<NX>;
  if (p.rpc < 1 || p.rpc > C::RPC_MAX) return cudaErrorInvalidValue;
  const int blocks = (p.rows_total + p.rpc - 1) / p.rpc;
  k_rk<T, NX><<<blocks, C::TPR * p.rpc, sizeof(cx<T>) * (size_t)p.rpc * C::FBUF, st>>>(p);
  return cudaGetLastError();
}

template <typename T, int NY>
cudaError_t launch_col_n(const ColParams& p, cudaStream_t st) {
  using C = ColCfg<NY>;
  const int blocks = (p.cols_total + C::CPB - 1) / C::CPB;
  if (p.nacc > 1)
    k_col<T, NY, 2><<<blocks, C::THREADS, col_smem<T, NY>(), st>>>(p);
  else
    k_col<T, NY, 1><<<blocks, C::THREADS, col_smem<T, NY>(), st>>>(p);
  return cudaGetLastError();
}

#define SBI_FOR_NX(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)
#define SBI_FOR_NY(X) X(1) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

template <typename T>
cudaError_t prepare_row_impl(int nx) {
  switch (nx) {
#define SBI_CASE(N) case N: return prepare_nx<T, N>();
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t prepare_col_impl(int ny) {
  switch (ny) {
#define SBI_CASE(N) case N: return prepare_ny<T, N>();
    SBI_FOR_NY(SBI_CASE)
#undef SBI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_row_impl(int nx, const RowParams& p, cudaStream_t st) {
  switch (nx) {
#define SBI_CASE(N) case N: return launch_row_n<T, N>(p, st);
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_rk_impl(int nx, const RkParams& p, cudaStream_t st) {
  switch (nx) {
#define SBI_CASE(N) case N: return launch_rk_n<T, N>(p, st);
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_col_impl(int ny, const ColParams& p, cudaStream_t st) {
  switch (ny) {
#define SBI_CASE(N) case N: return launch_col_n<T, N>(p, st);
    SBI_FOR_NY(SBI_CASE)
#undef SBI_CASE
    default: return cudaErrorInvalidValue;
  }
}

// Largest rows-per-block (power of two, <= the kernel's maximum) whose shared
// memory stays within 200 KB; 0 if even one row does not fit.
template <typename T>
int row_rpc_impl(int nx, int W, int nslots) {
  const size_t budget = 200 * 1024;
  int maxr = 0;
  size_t per = 0;
  switch (nx) {
#define SBI_CASE(N) case N: maxr = RowCfg<N>::RPC_MAX; per = row_smem<T, N>(1, W, nslots); break;
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return 0;
  }
  int tpr = 0;
  switch (nx) {
#define SBI_CASE(N) case N: tpr = RowCfg<N>::TPR; break;
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return 0;
  }
  int r = maxr;
  while (r > 1 && per * (size_t)r > budget) r /= 2;
  // a block must cover whole warps (the row FFTs synchronise whole warps)
  if (per * (size_t)r > budget || (r * tpr) % 32 != 0) return 0;
  return r;
}

}  // namespace sbi
