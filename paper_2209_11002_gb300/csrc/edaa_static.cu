// Allocation-free fit/loss evaluation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned
// by another allocator (for example a framework's caching pool that has
// reserved the whole GPU and forbids stray allocations), or a latency-bound
// loop that must never block in the driver's allocator.  For them this file
// offers a variant of the fit pass (the residual pass behind edaa_solve's
// fit and edaa_loss) whose per-CTA partial sums live in a fixed, file-scope
// device array instead of memory the library allocates.
//
// The array is g_fit_scratch below: kFitScratchDoubles doubles (384 KiB).  It
// is part of the library's device image, so every GPU that loads the library
// holds it until the process exits.  The image (all of the library's device
// code and this array) is loaded onto a device by the first call that needs
// it there: under CUDA's default lazy module loading, if this entry point is
// the first library call on a device, its set-up (the symbol lookup below)
// is what loads the image, and that takes device memory from the driver.
// A caller whose allocator later reserves the whole GPU must therefore make
// one library call on each device before that; a load that finds no memory
// is reported as EDAA_ERR_OOM.  All calls on a device share it and each
// call leaves its partials there; every slot the final reduction reads is
// written earlier in the same call, so nothing needs clearing between calls,
// but calls whose work overlaps on the GPU (different streams, or different
// host threads on one device) race on the array and must be serialised by
// the caller.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/edaa.h"

namespace edaa {
void set_last_error(const char* msg);  // the thread-local text behind edaa_last_error()
}

namespace {

constexpr int kFitThreads = 256;
constexpr int kFitMaxBlocks = 256;     // partial slots per run
constexpr int kFitMaxRuns = 64;        // runs per call
constexpr int kFitMaxP = 8;
constexpr int kFitMaxDevices = 64;
constexpr size_t kFitScratchDoubles = (size_t)kFitMaxBlocks * kFitMaxRuns * 3;  // 384 KiB

}  // namespace

static __device__ __align__(256) double g_fit_scratch[kFitScratchDoubles];

namespace {

edaa_status reject(edaa_status st, const char* msg) {
  edaa::set_last_error(msg);
  return st;
}

// Per pixel i and run m: r = x_i - E_m a_{m,i}; accumulates sum |r|, the
// largest per-pixel sum |r| (induced l1 norm) and sum r^2, then reduces the
// block's values per run in a fixed order into scratch[(block*M + m)*3 + k].
__global__ void __launch_bounds__(kFitThreads) k_fit_static_partial(const float* __restrict__ X, int L, int N, int p,
                                                                  int M, const float* __restrict__ E,
                                                                  const float* __restrict__ A, double* scratch) {
  __shared__ double red[3][kFitThreads];
  for (int m = 0; m < M; ++m) {
    const float* Em = E + (size_t)m * L * p;  // L x p row-major
    const float* Am = A + (size_t)m * p * N;  // p x N row-major
    double s1 = 0.0, s2 = 0.0, smax = 0.0;
    for (int i = blockIdx.x * kFitThreads + threadIdx.x; i < N; i += gridDim.x * kFitThreads) {
      float a[kFitMaxP];
      for (int j = 0; j < p; ++j) a[j] = Am[(size_t)j * N + i];
      const float* x = X + (size_t)i * L;
      float t1 = 0.f, t2 = 0.f;
      for (int l = 0; l < L; ++l) {
        float r = x[l];
        for (int j = 0; j < p; ++j) r = fmaf(-Em[l * p + j], a[j], r);
        t1 += fabsf(r);
        t2 = fmaf(r, r, t2);
      }
      s1 += (double)t1;
      s2 += (double)t2;
      smax = fmax(smax, (double)t1);
    }
    red[0][threadIdx.x] = s1;
    red[1][threadIdx.x] = smax;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = kFitThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[0][threadIdx.x] += red[0][threadIdx.x + w];
        red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
        red[2][threadIdx.x] += red[2][threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double* dst = scratch + ((size_t)blockIdx.x * M + m) * 3;
      dst[0] = red[0][0];
      dst[1] = red[1][0];
      dst[2] = red[2][0];
    }
    __syncthreads();
  }
}

__global__ void k_fit_static_reduce(const double* scratch, int blocks, int M, double* fit, double* fitmax,
                                    double* loss) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s1 = 0.0, smax = 0.0, s2 = 0.0;
  for (int b = 0; b < blocks; ++b) {
    const double* s = scratch + ((size_t)b * M + m) * 3;
    s1 += s[0];
    smax = fmax(smax, s[1]);
    s2 += s[2];
  }
  if (fit) fit[m] = s1;
  if (fitmax) fitmax[m] = smax;
  if (loss) loss[m] = s2;
}

std::mutex g_setup_mu;
void* g_scratch_ptr[kFitMaxDevices] = {};

// Device memory of the current device `dev` (or managed memory): a pointer to
// another GPU's memory would be read by kernels running on this one.
bool is_device_ptr(const void* p, int dev) {
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (pa.type == cudaMemoryTypeManaged) return true;
  return pa.type == cudaMemoryTypeDevice && pa.device == dev;
}

}  // namespace

extern "C" edaa_status edaa_fit_eval_static(const float* X, int L, int N, int p, int M, const float* E,
                                            const float* A, double* fit, double* fitmax, double* loss,
                                            void* stream) {
  if (!X || !E || !A) return reject(EDAA_ERR_ARG, "edaa_fit_eval_static: X, E and A are required");
  if (L < 1 || N < 1 || p < 1 || M < 1) return reject(EDAA_ERR_ARG, "edaa_fit_eval_static: L, N, p, M must be >= 1");
  if (p > kFitMaxP)
    return reject(EDAA_ERR_UNSUPPORTED, "edaa_fit_eval_static: p exceeds 8, the limit of this entry point");
  if (M > kFitMaxRuns)
    return reject(EDAA_ERR_UNSUPPORTED,
                  "edaa_fit_eval_static: M exceeds 64 runs, the size of its static scratch (call it per batch of runs)");
  if (!fit && !fitmax && !loss) return reject(EDAA_ERR_ARG, "edaa_fit_eval_static: no output requested");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return reject(EDAA_ERR_CUDA, "edaa_fit_eval_static: no CUDA device");
  }
  if (dev < 0 || dev >= kFitMaxDevices) return reject(EDAA_ERR_UNSUPPORTED, "edaa_fit_eval_static: device index");
  const void* ptrs[6] = {X, E, A, fit, fitmax, loss};
  for (const void* q : ptrs)
    if (q && !is_device_ptr(q, dev))
      return reject(EDAA_ERR_ARG,
                    "edaa_fit_eval_static: inputs and outputs must be device memory of the current device");
  void* scratch = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side
    // name g_fit_scratch is not a device address, so ask the runtime for it.
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_fit_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        // the lookup loads the library's device image when nothing has yet
        if (e == cudaErrorMemoryAllocation)
          return reject(EDAA_ERR_OOM, "edaa_fit_eval_static: no device memory to load the library's device code "
                                      "and static scratch (make one library call before reserving the GPU)");
        return reject(EDAA_ERR_CUDA, "edaa_fit_eval_static: cudaGetSymbolAddress of the static scratch failed");
      }
      g_scratch_ptr[dev] = ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  int blocks = (N + kFitThreads - 1) / kFitThreads;
  if (blocks > kFitMaxBlocks) blocks = kFitMaxBlocks;
  const cudaStream_t s = (cudaStream_t)stream;
  k_fit_static_partial<<<blocks, kFitThreads, 0, s>>>(X, L, N, p, M, E, A, (double*)scratch);
  k_fit_static_reduce<<<(M + 63) / 64, 64, 0, s>>>((const double*)scratch, blocks, M, fit, fitmax, loss);
  if (cudaGetLastError() != cudaSuccess) return reject(EDAA_ERR_CUDA, "edaa_fit_eval_static: launch failed");
  return EDAA_OK;
}
