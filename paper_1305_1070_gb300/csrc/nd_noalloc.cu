// Batched inversion of complex64 matrices in complex128 arithmetic that
// allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is
// frozen or owned by another allocator (a host framework that forbids device
// allocation inside its callbacks, or a fixed-footprint embedded service), or
// code that must not trigger the synchronisation an allocation can cause.
// This entry point serves them.  It is the root-block inversion of the
// single-precision paths (Gauss-Jordan with partial pivoting carried out in
// complex128 on a complex64 block), with the complex128 working copy held in a
// file-scope device array instead of a cudaMalloc'd workspace.

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "nd_gj.cuh"
#include "nd_internal.h"

namespace ndgf {
namespace {

// Working space: 2^18 complex128 elements (4 MiB), resident on every device
// that loads the library until the process exits.  batch * n * n <= 2^18, so
// the largest matrix is 512 x 512 (batch 1).
constexpr int64_t NOALLOC_ELEMS = int64_t(1) << 18;
constexpr int NOALLOC_MAX_N = 512;
__device__ __align__(256) double2 g_noalloc_work[NOALLOC_ELEMS];

// Device address of g_noalloc_work, looked up once per device (host code only
// sees a host-side stand-in under that name).
constexpr int MAX_DEVICES = 64;
double2* g_work_ptr[MAX_DEVICES];
cudaError_t g_work_err[MAX_DEVICES];
std::once_flag g_work_once[MAX_DEVICES];

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void k_invert_c64_noalloc(float2* A, int n, double2* work, int* n_singular) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nn = int64_t(n) * n;
  float2* M = A + int64_t(blockIdx.x) * nn;
  double2* W = work + int64_t(blockIdx.x) * nn;
  for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) W[i] = make_double2(double(M[i].x), double(M[i].y));
  __syncthreads();
  int* piv = reinterpret_cast<int*>(smem);
  const size_t colk_off = (size_t(n) * sizeof(int) + 15) & ~size_t(15);
  gj_invert<double>(W, n, n, piv, reinterpret_cast<double2*>(smem + colk_off), n_singular);
  for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) M[i] = make_float2(float(W[i].x), float(W[i].y));
}

}  // namespace
}  // namespace ndgf

using namespace ndgf;

extern "C" nd_status nd_invert_c64_noalloc(float* A, int32_t n, int32_t batch, int32_t* n_singular, void* stream) {
  if (!A || !n_singular) return fail(ND_ERR_INVALID_ARG, "nd_invert_c64_noalloc: NULL argument");
  if (n < 1 || n > NOALLOC_MAX_N || batch < 1)
    return fail(ND_ERR_INVALID_ARG, "nd_invert_c64_noalloc: need 1 <= n <= 512 and batch >= 1");
  if (int64_t(batch) * n * n > NOALLOC_ELEMS)
    return fail(ND_ERR_INVALID_ARG, "nd_invert_c64_noalloc: batch * n * n = " +
                                        std::to_string(int64_t(batch) * n * n) + " exceeds the fixed working space of " +
                                        std::to_string(NOALLOC_ELEMS) + " complex128 elements");
  if (!on_device(A) || !on_device(n_singular))
    return fail(ND_ERR_INVALID_ARG, "nd_invert_c64_noalloc: A and n_singular must be device arrays");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("nd_invert_c64_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(ND_ERR_UNSUPPORTED, "nd_invert_c64_noalloc: device index too large");
  std::call_once(g_work_once[dev], [dev] {
    g_work_err[dev] = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_work_ptr[dev]), g_noalloc_work);
  });
  if (g_work_err[dev] != cudaSuccess)
    return fail(ND_ERR_CUDA, std::string("nd_invert_c64_noalloc: cudaGetSymbolAddress: ") +
                                 cudaGetErrorString(g_work_err[dev]));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(n_singular, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("nd_invert_c64_noalloc: ") + cudaGetErrorString(e));
  const size_t shm = ((size_t(n) * sizeof(int) + 15) & ~size_t(15)) + size_t(n) * sizeof(double2);
  k_invert_c64_noalloc<<<batch, 256, shm, s>>>(reinterpret_cast<float2*>(A), n, g_work_ptr[dev], n_singular);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("nd_invert_c64_noalloc: ") + cudaGetErrorString(e));
  return ND_OK;
}
