// lr_truncate_noalloc: the rounding of lr_truncate with every piece of
// scratch memory in one file-scope device array instead of the handle's
// cudaMalloc'd workspace, and no handle at all (creating a handle allocates
// pinned host memory).
//
// Callers that cannot allocate: code that runs inside another framework's
// memory pool (a caching allocator owns the device memory and direct
// cudaMalloc calls would bypass its budget), and latency-critical loops where
// cudaMalloc may stall and cudaFree synchronises the whole device.  They pass
// their own inputs and outputs; the scratch below is reserved when the
// library is loaded and kept by every GPU that loads it until the process
// exits.
#include <mutex>

#include "lr_internal.h"

namespace lrp {
namespace {

constexpr int kStaticBlocks = 64;  // Gram partial sums: one per CTA
constexpr int kTileRows = 64;      // rows per Gram tile

// Scratch layout (doubles): Gram partials, two Gram matrices, Tc, Tr, the
// input weights, the status record.
constexpr size_t kOffPartial = 0;
constexpr size_t kOffGU = kOffPartial + (size_t)kStaticBlocks * KMAX * KMAX;
constexpr size_t kOffGV = kOffGU + (size_t)KMAX * KMAX;
constexpr size_t kOffTc = kOffGV + (size_t)KMAX * KMAX;
constexpr size_t kOffTr = kOffTc + (size_t)KMAX * KMAX;
constexpr size_t kOffW = kOffTr + (size_t)KMAX * KMAX;
constexpr size_t kOffState = kOffW + KMAX;
constexpr size_t kScratchDoubles = kOffState + (sizeof(SolveState) + 7) / 8;

// 2.2 MB of device memory per GPU, shared by every call on that GPU.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Per-device address of the scratch (host code must not use the symbol
// itself: on the host it is only a stand-in, not a device address).
double* g_scratch_ptr[64] = {};
cudaError_t g_scratch_err[64] = {};
std::once_flag g_scratch_once[64];

// G = X^T X, step 1: each of kStaticBlocks CTAs sums kTileRows-row tiles in
// a grid-stride loop (fixed order) into its own partial.
__global__ void __launch_bounds__(256) gram_static_partial(const double* __restrict__ X, int rows, int ld,
                                                           int k, double* __restrict__ scratch) {
  __shared__ double tile[kTileRows * KMAX];
  double* out = scratch + kOffPartial + (size_t)blockIdx.x * KMAX * KMAX;
  double acc[KMAX * KMAX / 256 + 1];
  const int npair = k * k;
#pragma unroll
  for (int j = 0; j < KMAX * KMAX / 256 + 1; ++j) acc[j] = 0.0;
  for (int r0 = blockIdx.x * kTileRows; r0 < rows; r0 += gridDim.x * kTileRows) {
    const int nr = min(kTileRows, rows - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTileRows * k; idx += blockDim.x) {
      const int i = idx % kTileRows, l = idx / kTileRows;
      tile[l * kTileRows + i] = i < nr ? X[(size_t)l * ld + r0 + i] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < KMAX * KMAX / 256 + 1; ++j) {
      const int idx = threadIdx.x + j * 256;
      if (idx < npair) {
        const int p = idx % k, q = idx / k;
        double s = 0.0;
        for (int i = 0; i < kTileRows; ++i) s += tile[p * kTileRows + i] * tile[q * kTileRows + i];
        acc[j] += s;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KMAX * KMAX / 256 + 1; ++j) {
    const int idx = threadIdx.x + j * 256;
    if (idx < npair) out[idx] = acc[j];
  }
}

// G = X^T X, step 2: sum the partials in block order.
__global__ void gram_static_sum(int k, double* __restrict__ scratch, size_t off_g) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < k * k; idx += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < kStaticBlocks; ++b) s += scratch[kOffPartial + (size_t)b * KMAX * KMAX + idx];
    const int p = idx % k, q = idx / k;
    scratch[off_g + p + (size_t)q * k] = s;
  }
}

// X[row, :R] = X[row, :k] Tm[:k, :R] in place: each thread keeps its row in
// shared memory, so writing the first R <= k columns cannot overwrite an
// input another thread still needs.
__global__ void __launch_bounds__(64) rotate_inplace(double* __restrict__ X, int rows, int ld, int k,
                                                     const double* __restrict__ scratch, size_t off_t) {
  __shared__ double row[64][KMAX + 1];
  const SolveState* st = reinterpret_cast<const SolveState*>(scratch + kOffState);
  const int R = st->rank;
  const double* tm = scratch + off_t;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows)
    for (int l = 0; l < k; ++l) row[threadIdx.x][l] = X[(size_t)l * ld + i];
  __syncthreads();
  if (i >= rows) return;
  for (int q = 0; q < R; ++q) {
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += row[threadIdx.x][l] * __ldg(&tm[l + (size_t)q * KMAX]);
    X[(size_t)q * ld + i] = s;
  }
}

}  // namespace
}  // namespace lrp

using namespace lrp;

extern "C" lr_status lr_truncate_noalloc(lr_mat* X, double eps, int rmax, void* cuda_stream) {
  if (!X) return LR_EINVAL;
  if (!(eps > 0.0) || eps >= 1.0 || rmax < 1) return LR_EINVAL;
  const int k = X->r;
  // The static scratch holds cores of at most KMAX = 64 columns.
  if (k < 1 || k > KMAX || X->rmax < k) return LR_EINVAL;
  if (X->n1 < 1 || X->n2 < 1 || X->ld < X->n1 || X->ld < X->n2) return LR_EINVAL;
  if (!X->U || !X->V || !X->s) return LR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(X->U) | reinterpret_cast<uintptr_t>(X->V) |
       reinterpret_cast<uintptr_t>(X->s)) & 15u)
    return LR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return LR_ECUDA; }
  // One-time set-up per device, with that device current.
  std::call_once(g_scratch_once[dev], [dev] {
    void* p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    g_scratch_ptr[dev] = static_cast<double*>(p);
  });
  if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) return LR_ECUDA;
  double* scratch = g_scratch_ptr[dev];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int keep_cap = rmax < X->rmax ? rmax : X->rmax;
  SolveState* state = reinterpret_cast<SolveState*>(scratch + kOffState);
  // The scratch keeps the previous call's contents: clear the status record.
  if (cudaMemsetAsync(state, 0, sizeof(SolveState), st) != cudaSuccess) return LR_ECUDA;
  if (cudaMemcpyAsync(scratch + kOffW, X->s, sizeof(double) * k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LR_ECUDA;
  gram_static_partial<<<kStaticBlocks, 256, 0, st>>>(X->U, X->n1, X->ld, k, scratch);
  gram_static_sum<<<(k * k + 255) / 256, 256, 0, st>>>(k, scratch, kOffGU);
  gram_static_partial<<<kStaticBlocks, 256, 0, st>>>(X->V, X->n2, X->ld, k, scratch);
  gram_static_sum<<<(k * k + 255) / 256, 256, 0, st>>>(k, scratch, kOffGV);
  if (cudaGetLastError() != cudaSuccess) return LR_ECUDA;
  CoreArgs<double> co;
  co.GC = scratch + kOffGU;
  co.GR = scratch + kOffGV;
  co.ldg = k;
  co.d = scratch + kOffW;
  co.k_dev = nullptr;
  co.k_host = k;
  co.eps = eps;
  co.rmax_out = keep_cap;
  co.Tc = scratch + kOffTc;
  co.Tr = scratch + kOffTr;
  co.s_out = X->s;
  co.st = state;
  if (launch_core<double>(co, false, st) != cudaSuccess) return LR_ECUDA;
  rotate_inplace<<<(X->n1 + 63) / 64, 64, 0, st>>>(X->U, X->n1, X->ld, k, scratch, kOffTc);
  rotate_inplace<<<(X->n2 + 63) / 64, 64, 0, st>>>(X->V, X->n2, X->ld, k, scratch, kOffTr);
  if (cudaGetLastError() != cudaSuccess) return LR_ECUDA;
  SolveState hs;
  if (cudaMemcpyAsync(&hs, state, sizeof(SolveState), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LR_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LR_ECUDA;
  X->r = hs.rank;
  if (hs.status) return static_cast<lr_status>(hs.status);
  return hs.cut ? LR_ENOCONV : LR_OK;
}
