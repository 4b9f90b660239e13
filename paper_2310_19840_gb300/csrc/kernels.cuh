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

#include "bank_model.h"
#include "fft.cuh"
#include "sbi_internal.h"

namespace sbi {

// ===========================================================================
// Row passes
// ===========================================================================
// Row-pass geometry: 8 elements per thread (radix-8 Stockham passes).  Up to
// n = 256 a row is transformed by one warp or less (warp-synchronous), longer
// rows by several warps with block barriers; a block holds up to 512
// threads.  In FP32 the blocks are compiled for two resident blocks per SM
// (64 registers per thread, no spills): measured against 16 elements per
// thread this doubles the warps per SM and runs the row passes faster at
// every size.
template <int NX>
struct RowCfg {
  static constexpr int n = NX / 2;                         // packed complex length
  static constexpr int R = cmin(8, n);   // elements per thread
  static constexpr int TPR = n / R;                        // threads per row
  static constexpr bool WARP = TPR <= 32;
  static constexpr int RPC_MAX = cmin(256, WARP ? cmax(16, 512 / TPR) : cmax(1, 512 / TPR));
  static constexpr int MAX_THREADS = TPR * RPC_MAX;
  static constexpr int FBUF = fft_scratch_len<n, R>();    // FFT scratch per row
  template <typename T>
  // 0: no minimum, the register count is left to the compiler
  static constexpr int min_blocks() { return sizeof(T) == 4 ? 2 : 0; }
};

// shared memory of a row block: per row the FFT scratch (row stride fbs), the
// physical slots and the staging row (stride sws) that receives the incoming
// mixed row.  The strides come from the bank model (bank_model.h).
template <typename T, int NX>
__host__ __device__ constexpr size_t row_smem(int rpc, int fbs, int sws, int nslots) {
  using C = RowCfg<NX>;
  return sizeof(cx<T>) * (size_t)rpc * ((size_t)fbs + (size_t)nslots * C::n + (size_t)sws);
}
// upper bound per row over every stride the bank model may pick
template <typename T, int NX>
__host__ __device__ constexpr size_t row_smem_bound(int W, int nslots) {
  constexpr int E = 128 / (int)sizeof(cx<T>);
  return row_smem<T, NX>(1, RowCfg<NX>::FBUF + E, W + E, nslots);
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

// Asynchronous copies global -> shared (cp.async, 8 or 16 bytes each): the
// copies of a whole staging pass are in flight together and land while the
// block computes; cp_async_wait_all + a block barrier make them visible.
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst_smem, const V* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(V) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk copies global -> shared by the tensor memory accelerator (TMA):
// cp.async.bulk moves a contiguous run (16-byte aligned ends, a multiple of 16
// bytes) and signals its completion on an mbarrier in shared memory as
// transaction bytes.  The barrier is armed with the expected byte count by
// mbarrier.arrive.expect_tx; a waiter polls mbarrier.try_wait.parity on the
// phase it expects, with an iteration limit after which it records a timeout
// in *flag and goes on (the host reports it; no kernel waits forever).
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// A wait gives up after one second of polling, or as soon as another thread
// has given up (the flag is read every 256 polls); it then records the
// timeout and waits once more, again for at most a second, for its copy.
// Returns false when it gave up: the caller issues and waits for nothing more.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int* flag) {
  if (mbar_try_wait(bar, parity)) return true;
  for (int round = 0; round < 2; ++round) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
      if (mbar_try_wait(bar, parity)) return round == 0;
      if ((it & 255u) == 0) {
        if (global_ns() - t0 > kWaitLimitNs) break;
        if (round == 0 && flag && *(volatile int*)flag) break;
      }
    }
    if (round == 0 && flag) atomicExch(flag, 1);
  }
  return false;
}

// Block-cooperative asynchronous load of one mixed buffer's rows into the
// staging rows stg[rl * sw + k], k < W; rows that are absent or inactive are
// zero-filled with plain stores.
template <typename T>
__device__ __forceinline__ void stage_async(cx<T>* stg_all, int sw, const BufRef& b, const RowIO& io) {
  using V = cx<T>;
  V* stg = stg_all + io.rl * sw;
  const V* src = reinterpret_cast<const V*>(b.ptr);
  for (int k = io.k0; k < io.W; k += io.kstep) {
    if (io.ok) cp_async_elem(stg + k, src + io.at(b, k));
    else stg[k] = mk<V>(T(0), T(0));
  }
  cp_async_commit();
}

// index of the first C2R op at or after o if it reads a single buffer (such
// inputs are staged asynchronously, ahead of time), else -1.  A C2R that sums
// several buffers is staged synchronously, so nothing may be in flight into
// the staging rows before it.
__device__ __forceinline__ int next_async_c2r(const RowParams& p, int o) {
  for (; o < p.nops; ++o)
    if (p.ops[o].kind == ROP_C2R) return p.ops[o].b == 1 ? o : -1;
  return -1;
}

// Packed inverse real FFT, input side, from the staged row: Z[k] = E + i O,
// E = X[k] + X*[n-k], O = (X[k] - X*[n-k]) e^{+2 pi i k / NX}, k = j + r TPR;
// X[k] = 0 for k >= W, and the Nyquist mode X[n] = 0.  The unnormalised
// inverse of Z gives NX * x packed as z[m] = x[2m] + i x[2m+1].  The function
// returns conj(Z): the inverse is taken as conj(F(conj Z)), so the caller runs
// the forward FFT and conjugates what it reads back.
template <typename T, int NX>
__device__ __forceinline__ void c2r_input(cx<T> (&x)[RowCfg<NX>::R], const cx<T>* stg, int W, int j,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  // e^{+2 pi i k / NX} = e^{+2 pi i j / NX} e^{+pi i r / R}: in FP32 with
  // R = 8 one table load and products by the 16th roots of unity
  constexpr bool kProd = C::R == 8 && kProductTwiddles<V>;
  const V wj = kProd ? cconj(__ldg(tw + tw_off(NX) + j)) : mk<V>(T(1), T(0));
  if (2 * W <= C::n) {
    // At most half the packed modes are kept: X[k] and X[n-k] are never both
    // nonzero, so Z[k] = X[k] (1 + i w) for k < W, conj(X[n-k]) (1 - i w) for
    // k > n - W and 0 in between (one load and one product per element).
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
      const int k = j + r * C::TPR;
      V w;
      if constexpr (kProd) w = r == 0 ? wj : cmul(wj, root16<1, V>(r));
      else w = cconj(__ldg(tw + tw_off(NX) + k));
      V z = mk<V>(T(0), T(0));
      if (k < W) z = cmul(stg[k], mk<V>(T(1) - w.y, w.x));                       // (1 + i w)
      else if (k > C::n - W) z = cmul(cconj(stg[C::n - k]), mk<V>(T(1) + w.y, -w.x));  // (1 - i w)
      x[r] = cconj(z);
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    const int k = j + r * C::TPR;
    const int kk = C::n - k;
    const V a = (k < W) ? stg[k] : mk<V>(T(0), T(0));
    const V b = (k > 0 && kk < W) ? stg[kk] : mk<V>(T(0), T(0));
    const V bc = cconj(b);
    const V E = cadd(a, bc);
    V w;
    if constexpr (kProd) w = r == 0 ? wj : cmul(wj, root16<1, V>(r));
    else w = cconj(__ldg(tw + tw_off(NX) + k));
    const V O = cmul(csub(a, bc), w);
    x[r] = cconj(cadd(E, rot<1>(O)));
  }
}

// Packed forward real FFT, output side, block-cooperative: each row's
// natural-order Z is in fb[rl]; the kept modes
// X[k] = 1/2 (Z[k] + Z*[n-k]) - i/2 e^{-2 pi i k / NX} (Z[k] - Z*[n-k]), k < W,
// are written to the transposed mixed field dst.
template <typename T, int NX>
__device__ __forceinline__ void r2c_store(const cx<T>* fb_all, int fbs, const BufRef& dst, const RowIO& io,
                                          const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  if (!io.ok) return;
  V* out = reinterpret_cast<V*>(dst.ptr);
  const V* fb = fb_all + io.rl * fbs;
  for (int k = io.k0; k < io.W; k += io.kstep) {
    const V zk = fb[pad(k)];
    const V zc = cconj(fb[pad((C::n - k) & (C::n - 1))]);
    const V s = cadd(zk, zc);
    const V d = cmul(csub(zk, zc), __ldg(tw + tw_off(NX) + k));
    out[io.at(dst, k)] = cscale(csub(s, rot<1>(d)), T(0.5));
  }
}

// Packed forward real FFT, output side, for rows whose transform ends in
// registers (kShuffleFft): thread j holds Z[j + r TPR] in x[r] and forms
// X[k] = 1/2 (Z[k] + Z*[n-k]) - i/2 e^{-2 pi i k / NX} (Z[k] - Z*[n-k]) for its
// own k = j + r TPR < W, writing it to the row's buffer xrow[k].  Z[n-k] sits
// in lane (TPR - j) mod TPR of the row, register R-1-r (thread 0: its own
// register (R - r) mod R), so one shuffle per kept register fetches it.  The
// twiddle is e^{-2 pi i j / NX} times e^{-2 pi i r / 16} (TPR / NX = 1/16)
// in FP32, the table entry in FP64.
template <typename T, int NX>
__device__ __forceinline__ void r2c_regs(const cx<T> (&x)[RowCfg<NX>::R], cx<T>* xrow, int W, int j,
                                         const cx<T>* __restrict__ tw) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int R = C::R, TPR = C::TPR;
  static_assert(R == 8 && 2 * R * TPR == NX, "rows of the shuffle-fed transforms only");
  constexpr bool kProd = kProductTwiddles<V>;     // FP64: every twiddle from the table
  const V wj = __ldg(tw + tw_off(NX) + j);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r * TPR >= W) break;                       // no thread keeps a mode here
    V zc;
    zc.x = __shfl_sync(0xffffffffu, x[R - 1 - r].x, (TPR - j) & (TPR - 1), TPR);
    zc.y = __shfl_sync(0xffffffffu, x[R - 1 - r].y, (TPR - j) & (TPR - 1), TPR);
    if (j == 0) zc = x[(R - r) & (R - 1)];
    zc = cconj(zc);
    const V zk = x[r];
    const int k = j + r * TPR;
    V w;
    if constexpr (kProd) w = r == 0 ? wj : cmul(wj, root16<-1, V>(r));
    else w = __ldg(tw + tw_off(NX) + k);
    const V sum = cadd(zk, zc);
    const V d = cmul(csub(zk, zc), w);
    if (k < W) xrow[k] = cscale(csub(sum, rot<1>(d)), T(0.5));
  }
}

// Block-cooperative store of the rows' kept modes xrow[k] (row stride fbs) to
// the transposed mixed field dst.
template <typename T>
__device__ __forceinline__ void store_modes(const cx<T>* x_all, int fbs, const BufRef& dst, const RowIO& io) {
  using V = cx<T>;
  if (!io.ok) return;
  V* out = reinterpret_cast<V*>(dst.ptr);
  const V* xr = x_all + io.rl * fbs;
  for (int k = io.k0; k < io.W; k += io.kstep) out[io.at(dst, k)] = xr[k];
}

template <typename T>
__device__ __forceinline__ T ipow(T v, int p) {
  T r = T(1);
  for (int i = 0; i < p; ++i) r *= v;
  return r;
}

template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<NX>::MAX_THREADS, RowCfg<NX>::template min_blocks<T>())
k_row(const __grid_constant__ RowParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = p.rpc;
  const int sw = p.sws;                            // staging row stride
  const int fbs = p.fbs;                           // FFT scratch row stride
  V* fb_all = reinterpret_cast<V*>(smem_raw);      // FFT scratch
  V* slot_base = fb_all + rpc * fbs;               // physical slots
  V* stg_all = slot_base + p.nslots * rpc * n;     // staging rows
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  V* fb = fb_all + rloc * fbs;
  const int row0 = p.row_begin + (int)blockIdx.x * rpc;
  const RowIO io(row0, rpc, p.rows_total, p.ny, p.W, p.active, p.member0);
  const int row = row0 + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row - member * p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);

  // eta is read through the L1 cache by every product of the row
  const V* eta = (act && p.eta.ptr) ? phys_row<T>(p.eta, member, y, NX) : nullptr;

  // the first single-buffer input is in flight from the start
  int pending = next_async_c2r(p, 0);
  if (pending >= 0) stage_async<T>(stg_all, sw, p.buf[p.ops[pending].a], io);

  for (int o = 0; o < p.nops; ++o) {
    const RowOp op = p.ops[o];
    V x[R];
    if (op.kind == ROP_C2R) {
      if (o == pending) {
        cp_async_wait_all();
        __syncthreads();  // every copy landed; scratch free (previous store done)
      } else {
        __syncthreads();  // staging and scratch free
        stage_mixed<T>(stg_all, sw, p.buf + op.a, op.b, io);
        __syncthreads();
      }
      c2r_input<T, NX>(x, stg_all + rloc * sw, p.W, fft_in_index<n, R>(j), tw);
      __syncthreads();  // every row has read its staging row; scratch free
      // the next single-buffer input lands while this one is transformed
      pending = next_async_c2r(p, o + 1);
      if (pending >= 0) stage_async<T>(stg_all, sw, p.buf[p.ops[pending].a], io);
    } else if (op.kind == ROP_PROD) {
      V* slot = op.slot == kNone ? nullptr : slot_base + (op.slot * rpc + rloc) * n;
      const T cf = T(op.coef);
      const bool running = (op.c & 2) != 0;
      const V* drow = (act && op.b > 0 && p.delta.ptr) ? phys_row<T>(p.delta, member, y, NX) : nullptr;
      const V* wrow = (act && (op.c & 1) && p.wgt.ptr) ? phys_row<T>(p.wgt, member, y, NX) : nullptr;
      const V* erow = op.a > 0 ? eta : nullptr;
      if (slot && erow && op.a == 1 && !drow && !wrow && running) {
        // the common running product slot <- eta * slot, straight-line
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int m = j + r * TPR;
          const V e = __ldg(erow + m);
          V v = slot[m];
          v = mk<V>(v.x * e.x, v.y * e.y);
          slot[m] = v;
          x[r] = mk<V>(cf * v.x, cf * v.y);
        }
      } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        V v = slot ? slot[m] : mk<V>(T(1), T(1));
        if (erow) {
          const V e = __ldg(erow + m);
          T e0 = e.x, e1 = e.y;
          for (int q = 1; q < op.a; ++q) { e0 *= e.x; e1 *= e.y; }
          v = mk<V>(v.x * e0, v.y * e1);
        }
        if (drow) {
          const V d = __ldg(drow + m);
          T d0 = d.x, d1 = d.y;
          for (int q = 1; q < op.b; ++q) { d0 *= d.x; d1 *= d.y; }
          v = mk<V>(v.x * d0, v.y * d1);
        }
        if (running && slot) slot[m] = v;
        if (wrow) {
          const V w = __ldg(wrow + m);
          v = mk<V>(v.x * w.x, v.y * w.y);
        }
        x[r] = mk<V>(cf * v.x, cf * v.y);
      }
      }
    } else {
      // ROP_N2 / ROP_WDOT / ROP_VFW: slots V (W for ROP_VFW), eta_x, [eta_y,] phi_x, [phi_y]
      const bool two_d = op.a == 2;
      const V* sV = slot_base + ((op.slot + 0) * rpc + rloc) * n;
      const V* sEx = slot_base + ((op.slot + 1) * rpc + rloc) * n;
      const V* sEy = two_d ? slot_base + ((op.slot + 2) * rpc + rloc) * n : nullptr;
      const V* sPx = slot_base + ((op.slot + (two_d ? 3 : 2)) * rpc + rloc) * n;
      const V* sPy = two_d ? slot_base + ((op.slot + 4) * rpc + rloc) * n : nullptr;
      const T g = T(op.coef);
      V* wout = (op.kind == ROP_WDOT && act) ? phys_row_w<T>(p.buf[op.dst], member, y, NX) : nullptr;
      const V* pgr = (op.kind == ROP_N2 && p.pg) ? reinterpret_cast<const V*>(p.pg) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V vv = sV[m], ex = sEx[m], px = sPx[m];
        const V ey = two_d ? sEy[m] : mk<V>(T(0), T(0));
        const V py = two_d ? sPy[m] : mk<V>(T(0), T(0));
        const V e = eta ? __ldg(eta + m) : mk<V>(T(0), T(0));
        const V pw = pgr ? __ldg(pgr + m) : mk<V>(T(0), T(0));
        T res[2];
        const T vc[2] = {vv.x, vv.y}, exc[2] = {ex.x, ex.y}, eyc[2] = {ey.x, ey.y};
        const T pxc[2] = {px.x, px.y}, pyc[2] = {py.x, py.y}, ec[2] = {e.x, e.y};
        const T pwc[2] = {pw.x, pw.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const T dot = exc[h] * pxc[h] + eyc[h] * pyc[h];
          const T ge2 = exc[h] * exc[h] + eyc[h] * eyc[h];
          const T gp2 = pxc[h] * pxc[h] + pyc[h] * pyc[h];
          const T num = vc[h] + dot;
          if (op.kind == ROP_N2)
            res[h] = -g * ec[h] + T(0.5) * (num * num / (T(1) + ge2) - gp2) - pwc[h];
          else if (op.kind == ROP_VFW)
            res[h] = vc[h] * (T(1) + ge2) - dot;
          else
            res[h] = num / (T(1) + ge2);
        }
        x[r] = mk<V>(res[0], res[1]);
        if (wout) wout[m] = x[r];
      }
      if (op.kind == ROP_WDOT) continue;
    }
    if (op.kind == ROP_C2R) {
      // inverse transform: the row in physical space, packed as complex
      // pairs; each thread's own elements m = j + r TPR come back in registers
      fft_regs_in_order<n, R, -1>(x, fb, j, tw);
      V* slot = slot_base + (op.slot * rpc + rloc) * n;
      V* out = (act && op.dst != kNone) ? phys_row_w<T>(p.buf[op.dst], member, y, NX) : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V z = cconj(x[r]);
        slot[m] = z;
        if (out) out[m] = z;
      }
      continue;
    }
    __syncthreads();  // scratch free (previous cooperative store done)
    if constexpr (kShuffleFft<n, R>) {
      // spectrum in registers, kept modes formed in the row's own threads
      fft_block_regs<n, R, -1>(x, fb, j, tw);
      r2c_regs<T, NX>(x, fb, p.W, j, tw);
      __syncthreads();  // every row's kept modes ready
      store_modes<T>(fb_all, fbs, p.buf[op.dst], io);
    } else {
      fft_to_smem<n, R, -1>(x, fb, j, tw);
      __syncthreads();  // every row's spectrum ready
      r2c_store<T, NX>(fb_all, fbs, p.buf[op.dst], io, tw);
    }
  }
}

// ===========================================================================
// State arithmetic.  The FP64 path keeps the state and the RK4 sums in double.
// The FP32 path keeps them as unevaluated sums hi + lo of two floats
// ("double-single", about 48 significant bits) updated with the error-free
// transformations TwoSum (Knuth) and FastTwoSum / the FMA product error
// (Dekker): on this GPU FP64 runs at a small fraction of the FP32 rate and an
// FP64 state update made the RK pass FP64-bound.  Both use 8 bytes per value.
// ===========================================================================
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add_f(FF x, float f) {
  FF s = ff_two_sum(x.hi, f);
  s.lo += x.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  FF s = ff_two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_mul_f(FF x, float f) {
  const float p = x.hi * f;
  float e = fmaf(x.hi, f, -p);
  e = fmaf(x.lo, f, e);
  return ff_fast_two_sum(p, e);
}
// product of two double-single values (the lo * lo term is below the result's
// last bit and dropped)
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return ff_fast_two_sum(p, e);
}


// A pair of state values (elements 2m, 2m+1) in one of the two storage
// formats: FP64, or double-single float pairs.  The FP64 format serves the
// FP64 path and, optionally, the FP32 path (its FP32 right-hand sides then
// accumulate into FP64 state and sums).  Inputs f are the working-precision
// stage values (float or double).
template <typename S> struct StatePair;
template <> struct StatePair<double> {
  double v[2];
  __device__ __forceinline__ static StatePair load(const void* base, int m) {
    const double2 d = reinterpret_cast<const double2*>(base)[m];
    return StatePair{{d.x, d.y}};
  }
  __device__ __forceinline__ void store(void* base, int m) const {
    reinterpret_cast<double2*>(base)[m] = make_double2(v[0], v[1]);
  }
  template <typename F> __device__ __forceinline__ void add(int h, F f) { v[h] += double(f); }
  // v += s * a (the RK4 update y + dt/6 (k1 + 2 k2 + 2 k3 + k4))
  __device__ __forceinline__ void add_scaled(int h, const StatePair& a, const RkScalar& s) {
    v[h] += s.d * a.v[h];
  }
  // the working copy of v + s f (a stage input) in the working precision T
  template <typename T, typename F>
  __device__ __forceinline__ T offset(int h, const RkScalar& s, F f) const {
    return T(v[h] + s.d * double(f));
  }
  __device__ __forceinline__ double value(int h) const { return v[h]; }
  __device__ __forceinline__ bool finite() const { return isfinite(v[0]) && isfinite(v[1]); }
  __device__ __forceinline__ static StatePair zero() { return StatePair{{0.0, 0.0}}; }
};
template <> struct StatePair<float> {
  FF v[2];
  __device__ __forceinline__ static StatePair load(const void* base, int m) {
    const float4 d = reinterpret_cast<const float4*>(base)[m];
    return StatePair{{FF{d.x, d.y}, FF{d.z, d.w}}};
  }
  __device__ __forceinline__ void store(void* base, int m) const {
    reinterpret_cast<float4*>(base)[m] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  }
  __device__ __forceinline__ void add(int h, float f) { v[h] = ff_add_f(v[h], f); }
  __device__ __forceinline__ void add_scaled(int h, const StatePair& a, const RkScalar& s) {
    v[h] = ff_add(v[h], ff_mul(a.v[h], FF{s.hi, s.lo}));
  }
  template <typename T>
  __device__ __forceinline__ T offset(int h, const RkScalar& s, float f) const {
    const FF r = ff_add(v[h], ff_mul_f(FF{s.hi, s.lo}, f));
    return T(r.hi + r.lo);
  }
  __device__ __forceinline__ float value(int h) const { return v[h].hi + v[h].lo; }
  __device__ __forceinline__ bool finite() const { return isfinite(v[0].hi) && isfinite(v[1].hi); }
  __device__ __forceinline__ static StatePair zero() { return StatePair{{FF{0.f, 0.f}, FF{0.f, 0.f}}}; }
};

// ===========================================================================
// RK4 stage pass (row layout).  State and sums in StatePair<T> storage.
// ===========================================================================
// RK stage geometry: blocks of kRkThreads threads (a whole row when a row
// needs more); three resident blocks per SM in FP32 (at most 85 registers),
// two in FP64 (128).
template <int NX>
struct RkCfg {
  static constexpr int RPC = cmax(1, kRkThreads / RowCfg<NX>::TPR);
  static constexpr int THREADS = RowCfg<NX>::TPR * RPC;
  template <typename T>
  static constexpr int min_blocks() { return sizeof(T) == 4 ? 3 : 2; }
};

// S: the state storage format (T itself, or double for the FP32 path with an
// FP64 state)
template <typename T, int NX, typename S>
__global__ void __launch_bounds__(RkCfg<NX>::THREADS, RkCfg<NX>::template min_blocks<T>())
k_rk(const __grid_constant__ RkParams p) {
  using V = cx<T>;
  using C = RowCfg<NX>;
  constexpr int n = C::n, R = C::R, TPR = C::TPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = p.rpc;
  V* fb_all = reinterpret_cast<V*>(smem_raw);
  const int fbs = p.fbs;                           // scratch row stride
  const int rloc = threadIdx.x / TPR, j = threadIdx.x % TPR;
  V* fb = fb_all + rloc * fbs;
  const int row0 = p.row_begin + (int)blockIdx.x * rpc;
  const RowIO io(row0, rpc, p.rows_total, p.ny, p.W, p.active, 0);
  const int row = row0 + rloc;
  const bool valid = row < p.rows_total;
  const int member = valid ? row / p.ny : 0;
  const int y = valid ? row - member * p.ny : 0;
  const bool act = valid && (p.active == nullptr || p.active[member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const long long off = (long long)y * NX;

  // new state in the working precision (the FFT inputs of the tail)
  using SP = StatePair<S>;
  V xe[R], xp[R];
  const long long eoff = member * p.eta0.stride + off, poff = member * p.phi0.stride + off;
  char* E0 = reinterpret_cast<char*>(p.eta0.ptr) + eoff * 8;   // 8 bytes per value
  char* P0 = reinterpret_cast<char*>(p.phi0.ptr) + poff * 8;
  bool bad = false;

  if (p.mode == RK_ENTRY) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = j + r * TPR;
      const SP e = act ? SP::load(E0, m) : SP::zero();
      const SP q = act ? SP::load(P0, m) : SP::zero();
      xe[r] = mk<V>(T(e.value(0)), T(e.value(1)));
      xp[r] = mk<V>(T(q.value(0)), T(q.value(1)));
    }
  } else {
    V x[R];
    // first inverse: phi~_t (stage) or the eta correction
    stage_mixed<T>(fb_all, fbs, &p.phit, 1, io);
    __syncthreads();
    c2r_input<T, NX>(x, fb, p.W, fft_in_index<n, R>(j), tw);
    row_group_sync<NX>();
    fft_regs_in_order<n, R, -1>(x, fb, j, tw);   // x[r]: element j + r TPR
    if (p.mode == RK_CORRECT || p.mode == RK_OFFSET) {
      const bool keep = p.mode == RK_CORRECT;   // RK_OFFSET leaves the state unchanged
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V c = cconj(x[r]);
        SP e = act ? SP::load(E0, m) : SP::zero();
        e.add(0, c.x);
        e.add(1, c.y);
        if (act && keep) e.store(E0, m);
        bad |= keep && !e.finite();
        xe[r] = mk<V>(T(e.value(0)), T(e.value(1)));
      }
      __syncthreads();
      stage_mixed<T>(fb_all, fbs, &p.corr_phi, 1, io);
      __syncthreads();
      c2r_input<T, NX>(x, fb, p.W, fft_in_index<n, R>(j), tw);
      row_group_sync<NX>();
      fft_regs_in_order<n, R, -1>(x, fb, j, tw);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V c = cconj(x[r]);
        SP q = act ? SP::load(P0, m) : SP::zero();
        q.add(0, c.x);
        q.add(1, c.y);
        if (act && keep) q.store(P0, m);
        bad |= keep && !q.finite();
        xp[r] = mk<V>(T(q.value(0)), T(q.value(1)));
      }
    } else {
      // classical RK4, y + dt/6 (k1 + 2 k2 + 2 k3 + k4): the sums take the
      // exact weights 1, 2, 2, 1; next-stage offsets c dt with c = (1/2, 1/2, 1).
      // dt/6 and c dt enter in the state's own format (double, or a
      // double-single pair), so the update never rounds the step to a float.
      const V* Vr = act ? phys_row<T>(p.V, member, y, NX) : nullptr;
      char* AE = reinterpret_cast<char*>(p.acc_eta.ptr) + (member * p.acc_eta.stride + off) * 8;
      char* AP = reinterpret_cast<char*>(p.acc_phi.ptr) + (member * p.acc_phi.stride + off) * 8;
      const T bw = T((p.stage == 1 || p.stage == 4) ? 1 : 2);
      const RkScalar cdt = p.cdt, dt6 = p.dt6;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * TPR;
        const V ft = cconj(x[r]);
        xe[r] = mk<V>(T(0), T(0));
        xp[r] = mk<V>(T(0), T(0));
        if (!act) continue;
        const V vv = Vr[m];
        SP ae = (p.stage > 1) ? SP::load(AE, m) : SP::zero();
        SP ap = (p.stage > 1) ? SP::load(AP, m) : SP::zero();
        ae.add(0, bw * vv.x);
        ae.add(1, bw * vv.y);
        ap.add(0, bw * ft.x);
        ap.add(1, bw * ft.y);
        SP e = SP::load(E0, m), q = SP::load(P0, m);
        if (p.stage < 4) {
          ae.store(AE, m);
          ap.store(AP, m);
          xe[r] = mk<V>(e.template offset<T>(0, cdt, vv.x), e.template offset<T>(1, cdt, vv.y));
          xp[r] = mk<V>(q.template offset<T>(0, cdt, ft.x), q.template offset<T>(1, cdt, ft.y));
        } else {
          e.add_scaled(0, ae, dt6);
          e.add_scaled(1, ae, dt6);
          q.add_scaled(0, ap, dt6);
          q.add_scaled(1, ap, dt6);
          e.store(E0, m);
          q.store(P0, m);
          bad |= !e.finite() || !q.finite();
          xe[r] = mk<V>(T(e.value(0)), T(e.value(1)));
          xp[r] = mk<V>(T(q.value(0)), T(q.value(1)));
        }
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
  fft_to_smem<n, R, -1>(xe, fb, j, tw);
  __syncthreads();
  r2c_store<T, NX>(fb_all, fbs, p.eta_hat, io, tw);
  __syncthreads();
  fft_to_smem<n, R, -1>(xp, fb, j, tw);
  __syncthreads();
  r2c_store<T, NX>(fb_all, fbs, p.phi_hat, io, tw);
}

// ===========================================================================
// Column pass: cpb columns per block (the size's CPB unless the launch asks
// for fewer), TPC threads per column, each column a contiguous run of NY
// complex.  Per column the block keeps the FFT scratch and the accumulators
// in shared memory; the per-mode multipliers come from tables in global
// memory (one real per stored mode and term).
// Inverse transforms use F^{-1}(X) = conj(F(conj X)) so one (forward) FFT
// instantiation serves both directions.
// ===========================================================================
// Column-pass geometry: 8 elements per thread (one warp per column at 256,
// two at 512, ...).  In FP32 columns of at least a warp are compiled for four
// resident blocks per SM (64 registers).

template <typename T, int NY>
struct ColCfg {
  static constexpr int RC = NY == 1 ? 1 : cmin(8, NY);
  static constexpr int TPC = NY / RC;
  static constexpr bool WARP = TPC <= 32;
  // 8-byte elements: 256 threads per block; 16-byte elements: half the columns
  static constexpr int CPB = NY == 1 ? 256 : cmax(1, 256 / TPC / (int)(sizeof(T) / 4));
  static constexpr int THREADS = TPC * CPB;
  // 512- to 2048-point columns by the split transforms of fft.cuh: forward
  // by decimation in frequency (natural loads, spectrum in decimated order),
  // inverse by decimation in time (decimated spectrum in, natural stores)
  static constexpr bool SPLIT = kSplitFft<NY, RC>;
  static constexpr int SCR = NY == 1 ? 0 : fft_scratch_len<NY, RC>();
  // accumulator length per column (padded where the modes are held with
  // stride NY / 256, so that those accesses spread over the banks)
  static constexpr int ACC = SPLIT ? padded_len(NY) : NY;
  static constexpr int MIN_BLOCKS = (sizeof(T) == 4 && RC == 8 && TPC >= 32) ? 4 : 0;  // 0: no minimum
};

template <typename T, int NY>
__host__ __device__ constexpr size_t col_smem(int nacc, int cpb) {
  using C = ColCfg<T, NY>;
  return sizeof(cx<T>) * (size_t)cpb * ((size_t)C::SCR + (size_t)C::ACC * nacc);
}
// the staged form adds, 128-byte aligned, one input column per column of the
// block (filled by a bulk copy) and one mbarrier per column
template <typename T, int NY>
__host__ __device__ constexpr size_t col_stage_offset(int nacc, int cpb) {
  return (col_smem<T, NY>(nacc, cpb) + 127) / 128 * 128;
}
template <typename T, int NY>
__host__ __device__ constexpr size_t col_smem_staged(int nacc, int cpb) {
  return col_stage_offset<T, NY>(nacc, cpb) + sizeof(cx<T>) * (size_t)cpb * NY + 8 * (size_t)cpb;
}
// columns long enough for bulk copies (whole 16-byte units, at least 256 bytes)
template <typename T, int NY>
inline constexpr bool kColStageable = NY >= 32;

// columns per block of a launch: the size's default CPB, or a smaller count
// that still makes whole warps (the column FFTs synchronise whole warps)
template <typename T, int NY>
__host__ __device__ constexpr int col_cpb(int requested) {
  using C = ColCfg<T, NY>;
  return requested > 0 ? requested : C::CPB;
}
template <typename T, int NY>
__host__ __device__ constexpr bool col_cpb_ok(int cpb) {
  using C = ColCfg<T, NY>;
  return cpb >= 1 && cpb <= C::CPB && (cpb * C::TPC) % 32 == 0;
}

template <typename V, typename S>
__device__ __forceinline__ V cmul_ipow(V x, S f, int q) {   // x f i^q
  const S re = x.x * f, im = x.y * f;
  S r2 = (q & 1) ? -im : re;
  S i2 = (q & 1) ? re : im;
  if (q & 2) {
    r2 = -r2;
    i2 = -i2;
  }
  return mk<V>(r2, i2);
}

// STAGED: each column's inputs arrive by bulk copies (TMA) into a staging
// column in shared memory, the next input in flight while the current one is
// transformed and accumulated; the arithmetic is that of the direct form.
template <typename T, int NY, bool STAGED>
__global__ void __launch_bounds__(ColCfg<T, NY>::THREADS, ColCfg<T, NY>::MIN_BLOCKS)
k_col(const __grid_constant__ ColParams p) {
  using V = cx<T>;
  using C = ColCfg<T, NY>;
  constexpr int RC = C::RC, TPC = C::TPC, SCR = C::SCR;
  const int cpb = col_cpb<T, NY>(p.cpb);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // staged form: the timeout flag, read first so that its latency overlaps
  // the set-up below
  const int gave_up = (STAGED && p.err_flag) ? *(volatile int*)p.err_flag : 0;
  const int c = threadIdx.x / TPC, j = threadIdx.x % TPC;
  V* base = reinterpret_cast<V*>(smem_raw);
  V* sc = base + c * SCR;                                   // FFT scratch
  V* acc0 = base + cpb * SCR + c * C::ACC * p.nacc;         // accumulators
  V* acc1 = acc0 + (p.nacc > 1 ? C::ACC : 0);
  const int gc = p.col_begin + (int)blockIdx.x * cpb + c;
  const bool valid = gc < p.cols_total;
  const int member = valid ? gc / p.W : 0;
  const int kx = valid ? gc % p.W : 0;
  const bool act = valid && (p.active == nullptr || p.active[p.member0 + member] != 0);
  const V* tw = reinterpret_cast<const V*>(p.tw);
  const long long col_off = (long long)kx * NY;

  // Slot r holds element nat(r) = j + r TPC of a column on input and on
  // output, and mode fwd(r) of its spectrum in between: the same for plain
  // transforms, the decimated order jd + r TPC for the split form.  acc_at:
  // position of a mode in the accumulators.
  constexpr bool SPLIT = C::SPLIT;
  const int jd = (NY / 256) * (j & 31) + (j >> 5);       // split: decimated lane order
  auto nat = [&](int r) { return j + r * TPC; };
  auto fwd = [&](int r) { return SPLIT ? jd + r * TPC : nat(r); };
  auto acc_at = [&](int m) { return SPLIT ? pad(m) : m; };
  // table position of slot r's mode m (split: the table's decimated order)
  auto tab_at = [&](int r, int m) { return SPLIT ? 256 * (j >> 5) + (j & 31) + 32 * r : m; };
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    acc0[acc_at(fwd(r))] = mk<V>(T(0), T(0));
    acc1[acc_at(fwd(r))] = mk<V>(T(0), T(0));
  }
  // staged form: the column's staging run and barrier; thread j = 0 of the
  // column arms the barrier and issues the copy of input i (16-byte aligned:
  // a column starts at a multiple of NY elements of its buffer)
  V* stg = nullptr;
  unsigned long long* bar = nullptr;
  constexpr unsigned kColBytes = (unsigned)(sizeof(V) * NY);
  auto issue = [&](int i) {
    const V* src = reinterpret_cast<const V*>(p.buf[i].ptr) + member * p.buf[i].stride + col_off;
    // the column's earlier reads of the staging run (generic proxy) come
    // before the copy that overwrites it (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, kColBytes + (unsigned)p.stall_tx);
    bulk_copy_g2s(stg, src, kColBytes, bar);
  };
  // live: the column's copies are issued and waited for; a launch that finds
  // the timeout flag already set (an earlier wait gave up) moves no data,
  // and a thread whose wait gave up issues and waits for nothing more
  bool live = act;
  if constexpr (STAGED) {
    unsigned char* st0 = smem_raw + col_stage_offset<T, NY>(p.nacc, cpb);
    stg = reinterpret_cast<V*>(st0) + c * NY;
    bar = reinterpret_cast<unsigned long long*>(st0 + sizeof(V) * (size_t)cpb * NY) + c;
    if (gave_up) live = false;
    if (j == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
    }
    __syncthreads();   // barriers initialised before any thread waits on them
    if (j == 0 && live && p.nin > 0) issue(0);
  }

  for (int i = 0; i < p.nin; ++i) {
    V x[RC];
    if constexpr (STAGED) {
      if (live) live = mbar_wait_bounded(bar, (unsigned)(i & 1), p.err_flag);
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = live ? stg[nat(r)] : mk<V>(T(0), T(0));
    } else {
      const V* src = reinterpret_cast<const V*>(p.buf[i].ptr) + member * p.buf[i].stride + col_off;
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = act ? src[nat(r)] : mk<V>(T(0), T(0));
    }
    if constexpr (SPLIT) {
      __syncthreads();        // scratch free (and, staged: the staging column read)
      if constexpr (STAGED) {
        if (j == 0 && live && i + 1 < p.nin) issue(i + 1);
      }
      fft_split_dif<NY, -1>(x, sc, j, tw);         // x[r]: mode fwd(r)
    } else if constexpr (NY > 1) {
      group_sync<C::WARP>();  // scratch free (and, staged: the staging column read)
      if constexpr (STAGED) {
        static_assert(C::WARP, "staged columns of the plain form fit one warp");
        if (j == 0 && live && i + 1 < p.nin) issue(i + 1);
      }
      fft_block_regs<NY, RC, -1>(x, sc, j, tw);   // x[r]: mode j + r TPC
    }
    for (int q = p.term_begin[i]; q < p.term_begin[i + 1]; ++q) {
      const ColTerm t = p.terms[q];
      const T* tab = reinterpret_cast<const T*>(t.tab) + col_off;
      const int ph = (t.gx + t.gy) & 3;
      V* acc = (t.acc == 0) ? acc0 : acc1;
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const int ni = fwd(r);
        const V v = x[r];
        acc[acc_at(ni)] = cadd(acc[acc_at(ni)], cmul_ipow(v, __ldg(tab + tab_at(r, ni)), ph));
      }
    }
  }
  // each thread reads back the modes it accumulated: no barrier
  for (int o = 0; o < p.nouts; ++o) {
    const ColTerm t = p.outs[o];
    const T* tab = reinterpret_cast<const T*>(t.tab) + col_off;
    const int ph = (t.gx + t.gy) & 3;
    const V* acc = (t.acc == 0) ? acc0 : acc1;
    V x[RC];
    // conjugated input: the forward FFT of conj(X) is the conjugate of F^{-1}(X)
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      const int ni = fwd(r);
      x[r] = cconj(cmul_ipow(acc[acc_at(ni)], __ldg(tab + tab_at(r, ni)), ph));
    }
    if constexpr (SPLIT) {
      __syncthreads();
      fft_split_dit<NY, -1>(x, sc, j, tw);         // x[r]: element nat(r)
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = cconj(x[r]);
    } else if constexpr (NY > 1) {
      group_sync<C::WARP>();
      fft_block_regs<NY, RC, -1>(x, sc, j, tw);
#pragma unroll
      for (int r = 0; r < RC; ++r) x[r] = cconj(x[r]);
    } else {
      x[0] = cconj(x[0]);
    }
    if (o == 0 && p.npass > 0 && act) {
      for (int q = 0; q < p.npass; ++q) {
        const V* ps = reinterpret_cast<const V*>(p.pass[q].ptr) + member * p.pass[q].stride + col_off;
#pragma unroll
        for (int r = 0; r < RC; ++r) x[r] = cadd(x[r], ps[nat(r)]);
      }
    }
    if (act) {
      V* dst = reinterpret_cast<V*>(p.buf[t.in].ptr) + member * p.buf[t.in].stride + col_off;
#pragma unroll
      for (int r = 0; r < RC; ++r) dst[nat(r)] = x[r];
    }
  }
}

// ---------------------------------------------------------------------------
// Multiplier tables: the real factor of a ColTerm for every stored mode
// (kx < W, all ny), evaluated in FP64 and rounded to the working precision.
// ---------------------------------------------------------------------------
// perm > 1: the column pass holds the modes of a column in the decimated
// order of the split transforms (mode n = perm (l + 32 r) + q read by lane l,
// warp q), so mode n is stored at (n mod perm) 256 + n / perm and the reads
// of a warp are contiguous.
template <typename T>
__global__ void k_coef_table(T* __restrict__ out, const TableSpec s, int perm) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)s.W * s.ny) return;
  const int kx = (int)(idx / s.ny), n = (int)(idx % s.ny);
  const long long at = (long long)kx * s.ny + (perm > 1 ? (n % perm) * 256 + n / perm : n);
  const int ns = (s.ny == 1) ? 0 : (n < s.ny / 2 ? n : n - s.ny);
  const double kxv = kx * s.two_pi_over_Lx, kyv = ns * s.two_pi_over_Ly;
  const double k = sqrt(kxv * kxv + kyv * kyv);
  double tk = 0.0, sk = 1.0;
  if (k > 0.0) {
    if (isinf(s.h0)) {
      tk = 1.0;
      sk = 0.0;
    } else {
      const double e = exp(-k * s.h0);
      tk = tanh(k * s.h0);
      sk = 2.0 * e / (1.0 + e * e);
    }
  }
  const double lam = s.filt_kf > 0.0 ? exp(-pow(k / s.filt_kf, s.filt_beta2)) : 1.0;
  double kp = 1.0;
  const int ap = s.kpow < 0 ? -s.kpow : s.kpow;
  for (int i = 0; i < ap; ++i) kp *= k;
  if (s.kpow < 0) kp = k > 0.0 ? 1.0 / kp : 0.0;
  double f = s.c * kp;
  double d = s.depth == 1 ? tk : (s.depth == 2 ? sk : (s.depth == 3 ? lam : 1.0));
  if (s.depth >= 8) {
    // factors of the implicit form of Appendix A: e_h = e^{-2 k h0}
    const double eh = isinf(s.h0) ? 0.0 : exp(-2.0 * k * s.h0);
    if (s.depth == 8) d = 1.0 + eh;
    else if (s.depth == 9) d = 1.0 - eh;
    else if (s.depth == 10) d = eh;
    else if (s.depth == 11) d = 1.0 / (1.0 + eh);
    else if (s.depth == 12) d = isinf(s.h0) ? 0.0 : exp(-k * s.h0);   // sqrt(e_h)
    else d = k > 0.0 ? 1.0 / (1.0 - eh) : 0.0;                          // D_h, 0 at k = 0
  } else if (s.depth >= 4) {
    // entries of e^{A tau}; cos - 1 as -2 sin^2(w tau / 2) (no cancellation)
    const double w = sqrt(s.gravity * k * tk);
    const double wt = w * s.tau, sh = sin(0.5 * wt);
    if (s.depth == 4) d = -2.0 * sh * sh;
    else if (s.depth == 5) d = k > 0.0 ? k * tk * sin(wt) / w : 0.0;
    else if (s.depth == 6) d = k > 0.0 ? s.gravity * sin(wt) / w : s.gravity * s.tau;
    else d = cos(wt);
  }
  for (int i = 0; i < s.gx; ++i) f *= kxv;
  for (int i = 0; i < s.gy; ++i) f *= kyv;
  const bool keep = kx < s.kx_keep && (ns < 0 ? -ns : ns) < s.ky_keep;
  if (s.mask == 2) f *= (keep ? d : 0.0) - 1.0;
  else f *= d * ((s.mask == 1 && !keep) ? 0.0 : 1.0);
  out[at] = T(f);
}

// order of the modes of a column in the multiplier tables (k_coef_table)
template <typename T>
int col_table_perm(int ny) {
  if (ny == 512 && ColCfg<T, 512>::SPLIT) return 2;
  if (ny == 1024 && ColCfg<T, 1024>::SPLIT) return 4;
  if (ny == 2048 && ColCfg<T, 2048>::SPLIT) return 8;
  return 1;
}

template <typename T>
cudaError_t launch_coef_table_impl(void* out, const TableSpec& s, cudaStream_t st) {
  const long long n = (long long)s.W * s.ny;
  k_coef_table<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<T*>(out), s,
                                                                 col_table_perm<T>(s.ny));
  return cudaGetLastError();
}

// Host-visible doubles <-> state storage of the working precision.
template <typename T>
__global__ void k_state_from_double(const double* __restrict__ src, void* __restrict__ dst, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if constexpr (sizeof(T) == 8) {
    reinterpret_cast<double*>(dst)[i] = src[i];
  } else {
    const float hi = float(src[i]);
    const float lo = float(src[i] - double(hi));
    reinterpret_cast<float2*>(dst)[i] = make_float2(hi, lo);
  }
}
template <typename T>
__global__ void k_state_to_double(const void* __restrict__ src, double* __restrict__ dst, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if constexpr (sizeof(T) == 8) {
    dst[i] = reinterpret_cast<const double*>(src)[i];
  } else {
    const float2 v = reinterpret_cast<const float2*>(src)[i];
    dst[i] = double(v.x) + double(v.y);
  }
}
template <typename T>
cudaError_t state_convert_impl(const void* src, void* dst, long long n, bool to_double, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (to_double) k_state_to_double<T><<<blocks, 256, 0, st>>>(src, reinterpret_cast<double*>(dst), n);
  else k_state_from_double<T><<<blocks, 256, 0, st>>>(reinterpret_cast<const double*>(src), dst, n);
  return cudaGetLastError();
}

// ===========================================================================
// Launchers
// ===========================================================================
template <typename T, int NX>
cudaError_t prepare_nx() {
  const int maxb = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_row<T, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rk<T, NX, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess || sizeof(T) == 8) return e;
  return cudaFuncSetAttribute(k_rk<T, NX, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
}

template <typename T, int NY>
cudaError_t prepare_ny() {
  cudaError_t e = cudaFuncSetAttribute(k_col<T, NY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)col_smem<T, NY>(kMaxColAcc, ColCfg<T, NY>::CPB));
  if (e != cudaSuccess || !kColStageable<T, NY>) return e;
  return cudaFuncSetAttribute(k_col<T, NY, kColStageable<T, NY>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)col_smem_staged<T, NY>(kMaxColAcc, ColCfg<T, NY>::CPB));
}

template <typename T, int NX>
cudaError_t launch_row_n(const RowParams& p, cudaStream_t st) {
  using C = RowCfg<NX>;
  if (p.rpc < 1 || p.rpc > C::RPC_MAX || p.row_begin < 0 || p.row_begin >= p.rows_total)
    return cudaErrorInvalidValue;
  const int blocks = (p.rows_total - p.row_begin + p.rpc - 1) / p.rpc;
  RowParams q = p;
  const bank::RowStrides rs =
      bank::choose(C::n, C::R, C::TPR, p.rpc, p.W, (int)sizeof(cx<T>), false, kShuffleFft<C::n, C::R>, C::FBUF);
  q.fbs = rs.fbs;
  q.sws = rs.sws;
  const size_t smem = row_smem<T, NX>(q.rpc, q.fbs, q.sws, q.nslots);
  if (smem > row_smem_bound<T, NX>(q.W, q.nslots) * (size_t)q.rpc) return cudaErrorInvalidValue;
  k_row<T, NX><<<blocks, C::TPR * q.rpc, smem, st>>>(q);
  return cudaGetLastError();
}

template <typename T, int NX>
cudaError_t launch_rk_n(const RkParams& p, cudaStream_t st) {
  using C = RowCfg<NX>;
  if (p.rpc < 1 || p.rpc > RkCfg<NX>::RPC || p.row_begin < 0 || p.row_begin >= p.rows_total)
    return cudaErrorInvalidValue;
  const int blocks = (p.rows_total - p.row_begin + p.rpc - 1) / p.rpc;
  RkParams q = p;
  q.fbs = bank::choose(C::n, C::R, C::TPR, p.rpc, p.W, (int)sizeof(cx<T>), true, false, C::FBUF).fbs;
  const size_t smem = sizeof(cx<T>) * (size_t)q.rpc * q.fbs;
  if (q.state64 && sizeof(T) == 4) k_rk<T, NX, double><<<blocks, C::TPR * q.rpc, smem, st>>>(q);
  else k_rk<T, NX, T><<<blocks, C::TPR * q.rpc, smem, st>>>(q);
  return cudaGetLastError();
}

template <typename T, int NY>
cudaError_t launch_col_n(const ColParams& p, cudaStream_t st) {
  using C = ColCfg<T, NY>;
  if (p.nacc < 1 || p.nacc > kMaxColAcc) return cudaErrorInvalidValue;
  const int cpb = col_cpb<T, NY>(p.cpb);
  if (!col_cpb_ok<T, NY>(cpb) || p.col_begin < 0 || p.col_begin >= p.cols_total) return cudaErrorInvalidValue;
  const int blocks = (p.cols_total - p.col_begin + cpb - 1) / cpb;
  if (p.staged) {
    if constexpr (kColStageable<T, NY>)
      k_col<T, NY, true><<<blocks, C::TPC * cpb, col_smem_staged<T, NY>(p.nacc, cpb), st>>>(p);
    else
      return cudaErrorInvalidValue;
  } else {
    k_col<T, NY, false><<<blocks, C::TPC * cpb, col_smem<T, NY>(p.nacc, cpb), st>>>(p);
  }
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
  // one block may take the whole 227 KB; blocks compiled for two per SM get
  // half of the SM's 228 KB less the 1 KB each block reserves
  size_t budget = 227 * 1024;
  int maxr = 0;
  size_t per = 0;
  switch (nx) {
#define SBI_CASE(N)                                                         \
  case N:                                                                   \
    maxr = RowCfg<N>::RPC_MAX;                                              \
    per = row_smem_bound<T, N>(W, nslots);                                  \
    if (RowCfg<N>::template min_blocks<T>() == 2) budget = 113 * 1024;      \
    break;
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

template <typename T>
int row_tpr_impl(int nx) {
  switch (nx) {
#define SBI_CASE(N) case N: return RowCfg<N>::TPR;
    SBI_FOR_NX(SBI_CASE)
#undef SBI_CASE
    default: return 0;
  }
}

template <typename T>
bool col_stageable_impl(int ny) {
  switch (ny) {
#define SBI_CASE(N) case N: return kColStageable<T, N>;
    SBI_FOR_NY(SBI_CASE)
#undef SBI_CASE
    default: return false;
  }
}

template <typename T>
int col_geometry_impl(int ny, int* tpc) {
  switch (ny) {
#define SBI_CASE(N) case N: *tpc = ColCfg<T, N>::TPC; return ColCfg<T, N>::CPB;
    SBI_FOR_NY(SBI_CASE)
#undef SBI_CASE
    default: *tpc = 0; return 0;
  }
}

}  // namespace sbi
