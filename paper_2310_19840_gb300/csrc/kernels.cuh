// kernels.cuh - row, column and RK4 passes of the ESBI step (templates).
//
// Included by the per-type instantiation units only.
#pragma once

#include <math.h>

#include "fft.cuh"
#include "sbi_internal.h"

namespace sbi {

// ===========================================================================
// Row passes: one group of TPR threads per row, RPC rows per block.
// ===========================================================================
template <int NX>
struct RowCfg {
  static constexpr int n = NX / 2;            // complex length of the packed real FFT
  static constexpr int R = cmin(8, n);        // elements per thread
  static constexpr int TPR = n / R;           // threads per row
  static constexpr int RPC = cmax(1, 256 / TPR);
  static constexpr int THREADS = TPR * RPC;
  static constexpr int FBUF = padded_len(n);  // padded FFT scratch per row (complex)
};

template <typename T, int NX>
__host__ __device__ constexpr size_t row_smem(int nslots) {
  using C = RowCfg<NX>;
  return sizeof(cx<T>) * (size_t)C::RPC * ((size_t)C::FBUF + (size_t)nslots * C::n);
}

template <typename T>
__device__ __forceinline__ const cx<T>* mixed_row(const BufRef& b, int member, int y, int W) {
  return reinterpret_cast<const cx<T>*>(b.ptr) + (long long)member * b.stride + (long long)y * W;
}
template <typename T>
__device__ __forceinline__ cx<T>* mixed_row_w(const BufRef& b, int member, int y, int W) {
  return reinterpret_cast<cx<T>*>(b.ptr) + (long long)member * b.stride + (long long)y * W;
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

// Packed inverse real FFT, input side: Z[k] = E[k] + i O[k] with
// E = X[k] + X*[n-k], O = (X[k] - X*[n-k]) e^{+2 pi i k / NX}, for the thread's
// k = j + r TPR.  X is the sum of `nb` mixed rows; X[k] = 0 for k >= W and the
// Nyquist mode X[n] = 0.  The unnormalised inverse then yields NX * x.
template <typename T, int NX>
__device__ __forceinline__ void c2r_input(cx<T> (&x)[RowCfg<NX>::R], const BufRef* bufs, int nb,
                                          int member, int y, int W, int j, bool act,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    const int k = j + r * C::TPR;
    V a = mk<V>(T(0), T(0)), b = mk<V>(T(0), T(0));
    if (act) {
      for (int q = 0; q < nb; ++q) {
        const V* src = mixed_row<T>(bufs[q], member, y, W);
        if (k < W) a = cadd(a, src[k]);
        const int kk = C::n - k;
        if (k > 0 && kk < W) b = cadd(b, src[kk]);
      }
    }
    const V bc = cconj(b);
    const V E = cadd(a, bc);
    const V O = cmul(csub(a, bc), cconj(__ldg(tw + tw_off(NX) + k)));
    x[r] = cadd(E, rot<1>(O));
  }
}

// Packed forward real FFT, output side: after the complex FFT of
// z[m] = x[2m] + i x[2m+1] the natural-order Z is in fb; the kept modes are
// X[k] = 1/2 (Z[k] + Z*[n-k]) - i/2 e^{-2 pi i k / NX} (Z[k] - Z*[n-k]), k < W.
template <typename T, int NX>
__device__ __forceinline__ void r2c_store(const cx<T>* fb, cx<T>* dst, int W, int j, bool act,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  if (!act) return;
  for (int k = j; k < W; k += C::TPR) {
    const V zk = fb[pad(k)];
    const V zc = cconj(fb[pad((C::n - k) & (C::n - 1))]);
    const V s = cadd(zk, zc);
    const V d = cmul(csub(zk, zc), __ldg(tw + tw_off(NX) + k));
    dst[k] = cscale(csub(s, rot<1>(d)), T(0.5));
  }
}

template <typename T>
__device__ __forceinline__ T ipow(T v, int p) {
  T r = T(1);
  for (int i = 0; i < p; ++i) r *= v;
  return r;
}

template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<NX>::THREADS)
k_row(const __grid_constant__ RowParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR, RPC = C::RPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* fb_all = reinterpret_cast<V*>(smem_raw);
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  V* fb = fb_all + rloc * C::FBUF;
  V* slot_base = fb_all + RPC * C::FBUF;
  const int row = blockIdx.x * RPC + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row % p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);

  V eta[R], del[R], wgt[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = j + r * TPR;
    eta[r] = (act && p.eta.ptr) ? phys_row<T>(p.eta, member, y, NX)[m] : mk<V>(T(0), T(0));
    del[r] = (act && p.delta.ptr) ? phys_row<T>(p.delta, member, y, NX)[m] : mk<V>(T(0), T(0));
    wgt[r] = (act && p.wgt.ptr) ? phys_row<T>(p.wgt, member, y, NX)[m] : mk<V>(T(0), T(0));
  }

  for (int o = 0; o < p.nops; ++o) {
    const RowOp op = p.ops[o];
    V x[R];
    if (op.kind == ROP_C2R) {
      c2r_input<T, NX>(x, p.buf + op.a, op.b, member, y, p.W, j, act, tw);
      __syncthreads();
      fft_block<n, R, +1>(x, fb, j, tw);
      V* slot = slot_base + (op.slot * RPC + rloc) * n;
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
      const V* slot = op.slot == kNone ? nullptr : slot_base + (op.slot * RPC + rloc) * n;
      const T cf = T(op.coef);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        V v = slot ? slot[m] : mk<V>(T(1), T(1));
        T f0 = cf * ipow(eta[r].x, op.a) * ipow(del[r].x, op.b) * ipow(wgt[r].x, op.c);
        T f1 = cf * ipow(eta[r].y, op.a) * ipow(del[r].y, op.b) * ipow(wgt[r].y, op.c);
        x[r] = mk<V>(f0 * v.x, f1 * v.y);
      }
    } else {
      // ROP_N2 / ROP_WDOT: slots V, eta_x, [eta_y,] phi_x, [phi_y]
      const bool two_d = op.a == 2;
      const V* sV = slot_base + ((op.slot + 0) * RPC + rloc) * n;
      const V* sEx = slot_base + ((op.slot + 1) * RPC + rloc) * n;
      const V* sEy = two_d ? slot_base + ((op.slot + 2) * RPC + rloc) * n : nullptr;
      const V* sPx = slot_base + ((op.slot + (two_d ? 3 : 2)) * RPC + rloc) * n;
      const V* sPy = two_d ? slot_base + ((op.slot + 4) * RPC + rloc) * n : nullptr;
      const T g = T(op.coef);
      V* wout = (op.kind == ROP_WDOT && act) ? phys_row_w<T>(p.buf[op.dst], member, y, NX) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V vv = sV[m], ex = sEx[m], px = sPx[m];
        const V ey = two_d ? sEy[m] : mk<V>(T(0), T(0));
        const V py = two_d ? sPy[m] : mk<V>(T(0), T(0));
        T res[2];
        const T vc[2] = {vv.x, vv.y}, exc[2] = {ex.x, ex.y}, eyc[2] = {ey.x, ey.y};
        const T pxc[2] = {px.x, px.y}, pyc[2] = {py.x, py.y}, ec[2] = {eta[r].x, eta[r].y};
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
    __syncthreads();
    fft_block<n, R, -1>(x, fb, j, tw);
    r2c_store<T, NX>(fb, act ? mixed_row_w<T>(p.buf[op.dst], member, y, p.W) : nullptr, p.W, j,
                     act, tw);
  }
}

// ===========================================================================
// RK4 stage pass (row layout).  FP64 state and sums for every real type.
// ===========================================================================
template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<NX>::THREADS)
k_rk(const __grid_constant__ RkParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR, RPC = C::RPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* fb = reinterpret_cast<V*>(smem_raw) + (threadIdx.x / TPR) * C::FBUF;
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  const int row = blockIdx.x * RPC + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row % p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const long long off = (long long)y * NX;

  double2 ye[R], yp[R];
  const double2* E0 = act ? reinterpret_cast<const double2*>(reinterpret_cast<const double*>(p.eta0.ptr) + member * p.eta0.stride + off) : nullptr;
  const double2* P0 = act ? reinterpret_cast<const double2*>(reinterpret_cast<const double*>(p.phi0.ptr) + member * p.phi0.stride + off) : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = j + r * TPR;
    ye[r] = act ? E0[m] : make_double2(0.0, 0.0);
    yp[r] = act ? P0[m] : make_double2(0.0, 0.0);
  }

  if (p.mode == RK_STAGE || p.mode == RK_CORRECT) {
    V x[R];
    // first inverse: phi~_t (stage) or the eta correction
    c2r_input<T, NX>(x, &p.phit, 1, member, y, p.W, j, act, tw);
    __syncthreads();
    fft_block<n, R, +1>(x, fb, j, tw);
    V f1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) f1[r] = fb[pad(j + r * TPR)];
    if (p.mode == RK_CORRECT) {
      c2r_input<T, NX>(x, &p.corr_phi, 1, member, y, p.W, j, act, tw);
      __syncthreads();
      fft_block<n, R, +1>(x, fb, j, tw);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const V c = fb[pad(j + r * TPR)];
        ye[r].x += double(f1[r].x); ye[r].y += double(f1[r].y);
        yp[r].x += double(c.x);     yp[r].y += double(c.y);
      }
    } else {
      const V* Vr = act ? phys_row<T>(p.V, member, y, NX) : nullptr;
      double2* AE = act ? reinterpret_cast<double2*>(reinterpret_cast<double*>(p.acc_eta.ptr) + member * p.acc_eta.stride + off) : nullptr;
      double2* AP = act ? reinterpret_cast<double2*>(reinterpret_cast<double*>(p.acc_phi.ptr) + member * p.acc_phi.stride + off) : nullptr;
      const double bw = (p.stage == 1 || p.stage == 4) ? (1.0 / 6.0) : (1.0 / 3.0);
      const double cn = (p.stage == 3) ? 1.0 : 0.5;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        if (!act) continue;
        const V vv = Vr[m];
        const double2 ke = make_double2(double(vv.x), double(vv.y));
        const double2 kp = make_double2(double(f1[r].x), double(f1[r].y));
        double2 ae, ap;
        if (p.stage == 1) {
          ae = make_double2(bw * ke.x, bw * ke.y);
          ap = make_double2(bw * kp.x, bw * kp.y);
        } else {
          ae = AE[m];
          ap = AP[m];
          ae.x += bw * ke.x; ae.y += bw * ke.y;
          ap.x += bw * kp.x; ap.y += bw * kp.y;
        }
        if (p.stage < 4) {
          AE[m] = ae;
          AP[m] = ap;
          ye[r].x += cn * p.dt * ke.x; ye[r].y += cn * p.dt * ke.y;
          yp[r].x += cn * p.dt * kp.x; yp[r].y += cn * p.dt * kp.y;
        } else {
          ye[r].x += p.dt * ae.x; ye[r].y += p.dt * ae.y;
          yp[r].x += p.dt * ap.x; yp[r].y += p.dt * ap.y;
        }
      }
    }
    const bool commit = (p.mode == RK_CORRECT) || (p.stage == 4);
    if (commit && act) {
      double2* E0w = reinterpret_cast<double2*>(reinterpret_cast<double*>(p.eta0.ptr) + member * p.eta0.stride + off);
      double2* P0w = reinterpret_cast<double2*>(reinterpret_cast<double*>(p.phi0.ptr) + member * p.phi0.stride + off);
      bool bad = false;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        E0w[m] = ye[r];
        P0w[m] = yp[r];
        bad |= !isfinite(ye[r].x) || !isfinite(ye[r].y) || !isfinite(yp[r].x) || !isfinite(yp[r].y);
      }
      if (bad && p.nonfinite) *p.nonfinite = 1;
    }
  }

  if (!p.tail) return;
  // working copies of the next stage: physical eta, mixed eta^ and phi^
  V x[R];
  V* ew = act ? phys_row_w<T>(p.eta_w, member, y, NX) : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    x[r] = mk<V>(T(ye[r].x), T(ye[r].y));
    if (ew) ew[j + r * TPR] = x[r];
  }
  __syncthreads();
  fft_block<n, R, -1>(x, fb, j, tw);
  r2c_store<T, NX>(fb, act ? mixed_row_w<T>(p.eta_hat, member, y, p.W) : nullptr, p.W, j, act, tw);
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = mk<V>(T(yp[r].x), T(yp[r].y));
  __syncthreads();
  fft_block<n, R, -1>(x, fb, j, tw);
  r2c_store<T, NX>(fb, act ? mixed_row_w<T>(p.phi_hat, member, y, p.W) : nullptr, p.W, j, act, tw);
}

// ===========================================================================
// Column pass: TX columns per block, TPC threads per column.
// ===========================================================================
template <int NY>
struct ColCfg {
  static constexpr int RC = NY >= 2048 ? 16 : cmin(8, NY);
  static constexpr int TPC = NY / RC;
  static constexpr int TX = NY == 1 ? 256 : cmax(1, cmin(64, 512 / TPC));
  static constexpr int THREADS = TPC * TX;
  static constexpr int CBUF = padded_len(NY);
};

template <typename T, int NY>
__host__ __device__ constexpr size_t col_smem() {
  return NY == 1 ? 16 : sizeof(cx<T>) * (size_t)ColCfg<NY>::TX * ColCfg<NY>::CBUF;
}

// c k^p D (i kx)^gx (i ky)^gy x  (negative powers of k vanish at k = 0)
template <typename T>
__device__ __forceinline__ cx<T> apply_term(const ColTerm& t, cx<T> x, T k, T kxv, T kyv, T tk,
                                            T sk, T lam) {
  using V = cx<T>;
  T f = T(t.c);
  if (t.kpow > 0) {
    f *= ipow(k, (int)t.kpow);
  } else if (t.kpow < 0) {
    f = (k > T(0)) ? f / ipow(k, -(int)t.kpow) : T(0);
  }
  if (t.depth == 1) f *= tk;
  else if (t.depth == 2) f *= sk;
  else if (t.depth == 3) f *= lam;
  f *= ipow(kxv, (int)t.gx) * ipow(kyv, (int)t.gy);
  V v = cscale(x, f);
  switch ((t.gx + t.gy) & 3) {
    case 1: v = rot<1>(v); break;
    case 2: v = mk<V>(-v.x, -v.y); break;
    case 3: v = rot<-1>(v); break;
    default: break;
  }
  return v;
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
  constexpr int RC = C::RC, TPC = C::TPC, TX = C::TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % TX, j = threadIdx.x / TX;
  V* sc = reinterpret_cast<V*>(smem_raw) + c * C::CBUF;
  const int gc = blockIdx.x * TX + c;
  const bool valid = gc < p.cols_total;
  const int member = valid ? gc / p.W : 0;
  const int kx = valid ? gc % p.W : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const bool deep = isinf(p.h0);
  const T h0 = deep ? T(0) : T(p.h0);
  const T kxv = T(kx) * T(p.two_pi_over_Lx);
  const T ky1 = T(p.two_pi_over_Ly);

  // depth factors of the thread's modes n = j + r TPC
  T tk[RC], sk[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    const int ni = j + r * TPC;
    const int ns = (NY == 1) ? 0 : (ni < NY / 2 ? ni : ni - NY);
    const T kyv = T(ns) * ky1;
    depth_factors<T>(sqrt(kxv * kxv + kyv * kyv), h0, deep, tk[r], sk[r]);
  }

  V acc[NACC][RC];
#pragma unroll
  for (int a = 0; a < NACC; ++a)
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[a][r] = mk<V>(T(0), T(0));
  const long long W = p.W;
  for (int i = 0; i < p.nin; ++i) {
    V x[RC];
    const V* src = reinterpret_cast<const V*>(p.buf[i].ptr) + member * p.buf[i].stride + kx;
#pragma unroll
    for (int r = 0; r < RC; ++r) x[r] = act ? src[(long long)(j + r * TPC) * W] : mk<V>(T(0), T(0));
    if constexpr (NY > 1) {
      __syncthreads();
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
        const V v = apply_term<T>(t, x[r], kk, kxv, kyv, tk[r], sk[r], T(1));
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
        x[r] = cscale(apply_term<T>(u, a, kk, kxv, kyv, tk[r], sk[r], lam), mfac);
      } else {
        x[r] = apply_term<T>(t, a, kk, kxv, kyv, tk[r], sk[r], lam);
        if (t.mask == 1 && !keep) x[r] = mk<V>(T(0), T(0));
      }
    }
    if constexpr (NY > 1) {
      __syncthreads();
      fft_block<NY, RC, +1>(x, sc, j, tw);
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = sc[pad(j + r * TPC)];
    }
    if (act) {
      V* dst = reinterpret_cast<V*>(p.buf[t.in].ptr) + member * p.buf[t.in].stride + kx;
#pragma unroll
      for (int r = 0; r < RC; ++r) dst[(long long)(j + r * TPC) * W] = x[r];
    }
  }
}

// ===========================================================================
// Launchers
// ===========================================================================
template <typename T, int NX>
cudaError_t prepare_nx() {
  cudaError_t e = cudaFuncSetAttribute(k_row<T, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)row_smem<T, NX>(kMaxSlots));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rk<T, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)row_smem<T, NX>(0));
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
  const int blocks = (p.rows_total + C::RPC - 1) / C::RPC;
  k_row<T, NX><<<blocks, C::THREADS, row_smem<T, NX>(p.nslots), st>>>(p);
  return cudaGetLastError();
}

template <typename T, int NX>
cudaError_t launch_rk_n(const RkParams& p, cudaStream_t st) {
  using C = RowCfg<NX>;
  const int blocks = (p.rows_total + C::RPC - 1) / C::RPC;
  k_rk<T, NX><<<blocks, C::THREADS, row_smem<T, NX>(0), st>>>(p);
  return cudaGetLastError();
}

template <typename T, int NY>
cudaError_t launch_col_n(const ColParams& p, cudaStream_t st) {
  using C = ColCfg<NY>;
  const int blocks = (p.cols_total + C::TX - 1) / C::TX;
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

template <typename T>
size_t row_smem_impl(int nx, int nslots) {
  switch (nx) {
#define SBI_CASE(N) case N: return row_smem<T, N>(nslots);
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return 0;
  }
}

}  // namespace sbi
