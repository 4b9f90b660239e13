// sbi_noalloc.cu - mass and energy of a state without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or a pre-sized arena, plugins that are handed device
// buffers but must not call cudaMalloc/cudaFree (which also synchronise the
// device), and hosts that forbid allocation after start-up.  For them
// sbi_invariants_noalloc computes the same two FP64 reductions as
// sbi_invariants from caller-owned device arrays, with its partial sums kept in
// one fixed, file-scope device array instead of context memory.
//
// The array lives in every process that loads the library, on every device it
// is used on, until the process exits.  All calls share it, so two calls whose
// work overlaps on the GPU (for example on two streams) race on it; callers
// must serialise them.  Nothing in it has to start at zero: every call writes
// each partial sum before reading it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/sbi.h"

namespace {

// Largest grid the entry point accepts: kNoallocMaxChunks chunks of
// kNoallocChunk points (2 * 4096 partial sums plus the two results: 64 KB).
constexpr int kNoallocChunk = 8192;
constexpr int kNoallocMaxChunks = 4096;
constexpr long long kNoallocMaxPoints = (long long)kNoallocChunk * kNoallocMaxChunks;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxChunks + 2];

// Device address of the scratch array per device, found once per device with
// that device current (the host-side symbol is not a device address).
double* g_scratch_ptr[kNoallocMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(double** out, const char** why) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    cudaGetLastError();
    *why = "no usable CUDA device";
    return SBI_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *why = "cudaGetSymbolAddress of the scratch array failed";
      return SBI_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SBI_OK;
}

// Partial sums of eta and 1/2 (phi V + g eta^2) over fixed chunks, each chunk
// reduced by one block in a fixed tree order (the same chunking and order as
// the context's reduction).
__global__ void k_partials(const double* __restrict__ eta, const double* __restrict__ phi,
                           const double* __restrict__ V, long long n, double g, double* __restrict__ part) {
  __shared__ double sm[2][256];
  const long long base = (long long)blockIdx.x * kNoallocChunk;
  double m = 0.0, e = 0.0;
  for (int i = threadIdx.x; i < kNoallocChunk; i += blockDim.x) {
    const long long q = base + i;
    if (q < n) {
      const double h = eta[q];
      m += h;
      e += 0.5 * (phi[q] * V[q] + g * h * h);
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
    part[2 * blockIdx.x] = sm[0][0];
    part[2 * blockIdx.x + 1] = sm[1][0];
  }
}

// Sum of the chunk partials in chunk order by one thread (deterministic), then
// scaled by the cell area; results at part[2 * kNoallocMaxChunks + {0, 1}].
__global__ void k_total(double* __restrict__ part, int nchunks, double dA) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = 0.0, e = 0.0;
  for (int q = 0; q < nchunks; ++q) {
    m += part[2 * q];
    e += part[2 * q + 1];
  }
  part[2 * kNoallocMaxChunks] = m * dA;
  part[2 * kNoallocMaxChunks + 1] = e * dA;
}

thread_local char g_noalloc_err[256] = "no error";

int noalloc_fail(int code, const char* msg) {
  std::snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg);
  return code;
}

}  // namespace

extern "C" {

int sbi_invariants_noalloc(const sbi_grid* g, double gravity, const double* eta, const double* phi,
                           const double* V, void* cuda_stream, double* mass, double* energy) {
  if (!g || !eta || !phi || !V || !mass || !energy)
    return noalloc_fail(SBI_EINVAL, "sbi_invariants_noalloc: NULL argument");
  if (g->nx < 1 || g->ny < 1 || !(g->Lx > 0.0) || (g->ny > 1 && !(g->Ly > 0.0)))
    return noalloc_fail(SBI_EINVAL, "sbi_invariants_noalloc: bad grid");
  if (!(gravity > 0.0)) return noalloc_fail(SBI_EINVAL, "sbi_invariants_noalloc: gravity must be > 0");
  const long long n = (long long)g->nx * g->ny;
  if (n > kNoallocMaxPoints)
    return noalloc_fail(SBI_EINVAL,
                        "sbi_invariants_noalloc: grid larger than the 33554432-point limit of the "
                        "static scratch array");
  double* scratch = nullptr;
  const char* why = nullptr;
  int rc = scratch_for_current_device(&scratch, &why);
  if (rc) return noalloc_fail(rc, why);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nchunks = (int)((n + kNoallocChunk - 1) / kNoallocChunk);
  const double Ly = g->ny > 1 ? g->Ly : 1.0;
  const double dA = (g->Lx / g->nx) * (Ly / g->ny);
  k_partials<<<nchunks, 256, 0, st>>>(eta, phi, V, n, gravity, scratch);
  k_total<<<1, 32, 0, st>>>(scratch, nchunks, dA);
  double res[2] = {0.0, 0.0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res, scratch + 2 * kNoallocMaxChunks, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(SBI_ECUDA, cudaGetErrorString(e));
  }
  *mass = res[0];
  *energy = res[1];
  return SBI_OK;
}

const char* sbi_noalloc_last_error(void) { return g_noalloc_err; }

}  // extern "C"
