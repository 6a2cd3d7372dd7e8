// Device pieces of the self-consistent Schroedinger-Poisson loop: the
// five-point Poisson operator of a rectangular grid and its direct solver,
// and the two vector operations of the Newton-Krylov iteration.  The paper
// motivates the diagonal of G^< by the electron density that enters Poisson's
// equation (Sec. 1); the electrostatics itself is not in the paper.
//
// Grid: nx (transport) x ny (transverse), site (x, y) = x * ny + y.
//   (K u)_j = sum_{k neighbour of j} (u_j - u_k)
// with u = 0 on ghost columns x = -1 and x = nx (Dirichlet at the ends) and
// no neighbours across y = 0, ny - 1 (Neumann at the edges).  K = Kx (x) I +
// I (x) Ky, Kx = tridiag(-1, 2, -1), Ky the path Laplacian with free ends,
// whose eigenvectors are the cosines q_k(y) = c_k cos(k pi (y + 1/2) / ny)
// (c_0 = 1 / sqrt(ny), else sqrt(2 / ny)) with eigenvalues 2 - 2 cos(k pi / ny).
// The solver of (K + shift I) u = rhs transforms along y, solves one
// tridiagonal system per mode along x (Thomas algorithm), and transforms back.

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "nd_internal.h"

using namespace ndgf;

struct nd_poisson {
  int nx = 0, ny = 0;
  double* d_Q = nullptr;     // [ny][ny]: Q[y][k]
  double* d_mu = nullptr;    // [ny]: eigenvalues 2 - 2 cos(k pi / ny) of Ky
  double* d_work = nullptr;  // [batch][nx][ny] transformed right-hand sides, then [batch][ny][nx] Thomas factors
  int work_batch = 0;
  ~nd_poisson() {
    cudaFree(d_Q);
    cudaFree(d_mu);
    cudaFree(d_work);
  }
};

namespace {

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void k_poisson_apply(const double* __restrict__ u, double* __restrict__ out, int nx, int ny) {
  const int64_t n = int64_t(nx) * ny;
  const int64_t b = blockIdx.y;
  const double* U = u + b * n;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(j / ny), y = int(j % ny);
    const double uj = U[j];
    double r = 2.0 * uj;  // the two transport neighbours (ghosts at the ends are 0)
    if (x > 0) r -= U[j - ny];
    if (x + 1 < nx) r -= U[j + ny];
    if (y > 0) r += uj - U[j - 1];
    if (y + 1 < ny) r += uj - U[j + 1];
    out[b * n + j] = r;
  }
}

// w[b][x][k] = sum_y Q[y][k] r[b][x][y]   (transpose = 0), or
// u[b][x][y] = sum_k Q[y][k] w[b][x][k]   (transpose = 1)
__global__ void k_poisson_transform(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ Q,
                                    int nx, int ny, int back) {
  const int64_t n = int64_t(nx) * ny;
  const int64_t b = blockIdx.y;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(j / ny), i = int(j % ny);
    const double* row = in + b * n + int64_t(x) * ny;
    double s = 0.0;
    if (!back)
      for (int y = 0; y < ny; ++y) s += Q[int64_t(y) * ny + i] * row[y];
    else
      for (int k = 0; k < ny; ++k) s += Q[int64_t(i) * ny + k] * row[k];
    out[b * n + j] = s;
  }
}

// Per mode k: (Kx + mu_k + shift) v = w along x, Thomas algorithm in place on
// w.  With the off-diagonals -1 and the diagonal b: g_x = 1 / (b - g_{x-1})
// (g_{-1} = 0, g_x <= 1 because b >= 2), forward d'_x = (d_x + d'_{x-1}) g_x,
// back v_x = d'_x + g_x v_{x+1}; the g_x of the mode are kept in gbuf.
__global__ void k_poisson_modes(double* __restrict__ w, double* __restrict__ gbuf, const double* __restrict__ mu,
                                double shift, int nx, int ny) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ny) return;
  double* W = w + int64_t(blockIdx.y) * nx * ny;
  double* g = gbuf + (int64_t(blockIdx.y) * ny + k) * nx;
  const double b = 2.0 + mu[k] + shift;
  double prev = 0.0, gp = 0.0;
  for (int x = 0; x < nx; ++x) {
    const double gx = 1.0 / (b - gp);
    g[x] = gx;
    const double v = (W[int64_t(x) * ny + k] + prev) * gx;
    W[int64_t(x) * ny + k] = v;
    prev = v;
    gp = gx;
  }
  double next = 0.0;
  for (int x = nx - 1; x >= 0; --x) {
    const double v = W[int64_t(x) * ny + k] + (x + 1 < nx ? g[x] : 0.0) * next;
    W[int64_t(x) * ny + k] = v;
    next = v;
  }
}

// Deterministic dot product: fixed grid of partial sums, then one CTA.
constexpr int DOT_BLOCKS = 256;
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    s = fma(x[i], y[i], s);
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
__global__ void k_dot_final(const double* part, double* out) {
  __shared__ double red[DOT_BLOCKS];
  red[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int h = DOT_BLOCKS / 2; h > 0; h >>= 1) {
    if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

__global__ void k_vmul(const double* __restrict__ d, const double* __restrict__ x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = d[i] * x[i];
}

__global__ void k_scale_pos(double a, const double* __restrict__ x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = fmax(0.0, a * x[i]);
}

double* g_dot_part[64] = {};

}  // namespace

extern "C" nd_status nd_poisson_create(int32_t nx, int32_t ny, nd_poisson** out) {
  if (!out || nx < 1 || ny < 1) return fail(ND_ERR_INVALID_ARG, "nd_poisson_create: bad argument");
  *out = nullptr;
  std::vector<double> Q(size_t(ny) * ny), mu(ny);
  for (int y = 0; y < ny; ++y)
    for (int k = 0; k < ny; ++k)
      Q[size_t(y) * ny + k] = (k == 0 ? std::sqrt(1.0 / ny) : std::sqrt(2.0 / ny)) * std::cos(k * M_PI * (y + 0.5) / ny);
  for (int k = 0; k < ny; ++k) mu[k] = 2.0 - 2.0 * std::cos(k * M_PI / ny);
  auto P = new nd_poisson();
  P->nx = nx;
  P->ny = ny;
  auto up = [](const std::vector<double>& h, double** d) {
    if (cudaMalloc((void**)d, h.size() * sizeof(double)) != cudaSuccess) return false;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(Q, &P->d_Q) || !up(mu, &P->d_mu)) {
    cudaGetLastError();
    delete P;
    return fail(ND_ERR_OOM, "nd_poisson_create: device allocation failed");
  }
  *out = P;
  return ND_OK;
}

extern "C" void nd_poisson_destroy(nd_poisson* P) { delete P; }

extern "C" nd_status nd_poisson_apply(nd_poisson* P, const double* u, double* out, int32_t batch, void* stream) {
  if (!P || batch < 1 || !on_device(u) || !on_device(out))
    return fail(ND_ERR_INVALID_ARG, "nd_poisson_apply: bad argument (arrays must be device pointers)");
  const int64_t n = int64_t(P->nx) * P->ny;
  k_poisson_apply<<<dim3(unsigned(std::min<int64_t>((n + 255) / 256, 4096)), batch), 256, 0, (cudaStream_t)stream>>>(
      u, out, P->nx, P->ny);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_poisson_apply: ") + cudaGetErrorString(e));
}

extern "C" nd_status nd_poisson_solve(nd_poisson* P, double shift, const double* rhs, double* u, int32_t batch,
                                      void* stream) {
  if (!P || batch < 1 || !(shift >= 0.0) || !on_device(rhs) || !on_device(u))
    return fail(ND_ERR_INVALID_ARG, "nd_poisson_solve: bad argument (shift >= 0, arrays must be device pointers)");
  const int64_t n = int64_t(P->nx) * P->ny;
  if (batch > P->work_batch) {
    cudaFree(P->d_work);
    P->d_work = nullptr;
    P->work_batch = 0;
    if (cudaMalloc((void**)&P->d_work, size_t(2 * n) * batch * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ND_ERR_OOM, "nd_poisson_solve: cannot allocate the work array");
    }
    P->work_batch = batch;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 g(unsigned(std::min<int64_t>((n + 255) / 256, 4096)), batch);
  double* w = P->d_work;
  double* gb = P->d_work + n * batch;
  k_poisson_transform<<<g, 256, 0, s>>>(rhs, w, P->d_Q, P->nx, P->ny, 0);
  k_poisson_modes<<<dim3((P->ny + 63) / 64, batch), 64, 0, s>>>(w, gb, P->d_mu, shift, P->nx, P->ny);
  k_poisson_transform<<<g, 256, 0, s>>>(w, u, P->d_Q, P->nx, P->ny, 1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_poisson_solve: ") + cudaGetErrorString(e));
}

extern "C" nd_status nd_vec_dot(const double* x, const double* y, int64_t n, double* out, void* stream) {
  if (n < 0 || !on_device(x) || !on_device(y) || !on_device(out))
    return fail(ND_ERR_INVALID_ARG, "nd_vec_dot: bad argument (arrays must be device pointers)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(ND_ERR_CUDA, "nd_vec_dot: no device");
  if (!g_dot_part[dev] && cudaMalloc((void**)&g_dot_part[dev], DOT_BLOCKS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ND_ERR_OOM, "nd_vec_dot: cannot allocate the partial sums");
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_dot_partial<<<DOT_BLOCKS, 256, 0, s>>>(x, y, n, g_dot_part[dev]);
  k_dot_final<<<1, DOT_BLOCKS, 0, s>>>(g_dot_part[dev], out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_vec_dot: ") + cudaGetErrorString(e));
}

extern "C" nd_status nd_vec_axpby(double a, const double* x, double b, double* y, int64_t n, void* stream) {
  if (n < 0 || !on_device(x) || !on_device(y))
    return fail(ND_ERR_INVALID_ARG, "nd_vec_axpby: bad argument (arrays must be device pointers)");
  if (n == 0) return ND_OK;
  k_axpby<<<unsigned(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, (cudaStream_t)stream>>>(a, x, b, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_vec_axpby: ") + cudaGetErrorString(e));
}

extern "C" nd_status nd_vec_mul(const double* d, const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || !on_device(d) || !on_device(x) || !on_device(y))
    return fail(ND_ERR_INVALID_ARG, "nd_vec_mul: bad argument (arrays must be device pointers)");
  if (n == 0) return ND_OK;
  k_vmul<<<unsigned(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, (cudaStream_t)stream>>>(d, x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_vec_mul: ") + cudaGetErrorString(e));
}

extern "C" nd_status nd_vec_scale_pos(double a, const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || !on_device(x) || !on_device(y))
    return fail(ND_ERR_INVALID_ARG, "nd_vec_scale_pos: bad argument (arrays must be device pointers)");
  if (n == 0) return ND_OK;
  k_scale_pos<<<unsigned(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, (cudaStream_t)stream>>>(a, x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ND_OK : fail(ND_ERR_CUDA, std::string("nd_vec_scale_pos: ") + cudaGetErrorString(e));
}
