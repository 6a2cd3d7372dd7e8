// Input checks of nd_factor and nd_diag_green.
//
// The fold and the extraction rely on two properties of the inputs:
//  - A = (E + i eta) I - H - Sigma^r is complex symmetric (A = A^T), which
//    the LDL^T-type elimination of paper Sec. 3.1 uses when it stores one of
//    A_iB / A_Bi and one of G_IB / G_BI (G^r = (G^r)^T);
//  - Sigma^< and Sigma^> are skew-Hermitian (paper Sec. 3.1, the three-cluster
//    G^< formulas: the P_BI = -(P_IB)^dagger step).
// H must therefore have symmetric values on its (structurally symmetric)
// pattern, every contact block Sigma^r_c must be complex symmetric, and every
// contact block of Sigma^< / Sigma^> and the phonon diagonals must be
// skew-Hermitian.  Host arrays are checked on the host before any device work
// (the call fails with the status); device arrays are checked by a kernel on
// the call's stream, which records the failure for nd_fact_status.
//
// Tolerance ND_INPUT_TOL, relative: for H, |H_jk - H_kj| <= tol max(|H_jk|,
// |H_kj|); for a contact block S (per energy), |S_ab -/+ S_ba| <= tol max|S|;
// for a phonon diagonal s_j, |Re s_j| <= tol |s_j|.  Non-finite values fail.

#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "nd_check.h"

namespace ndgf {

const int32_t* csr_transpose(const nd_plan* p) { return p->csr_T.data(); }

namespace {

bool close_sym(double a, double b, double scale) { return std::fabs(a - b) <= ND_INPUT_TOL * scale; }

// Host: one contact block of one energy, symmetric (skew = false) or
// skew-Hermitian (skew = true).
bool host_block_ok(const double* S, int m, bool skew) {
  double mx = 0.0;
  for (int64_t q = 0; q < int64_t(m) * m; ++q) {
    const double a = std::hypot(S[2 * q], S[2 * q + 1]);
    if (!std::isfinite(a)) return false;
    mx = std::max(mx, a);
  }
  for (int a = 0; a < m; ++a)
    for (int b = a; b < m; ++b) {
      const double* x = S + 2 * (int64_t(a) * m + b);
      const double* y = S + 2 * (int64_t(b) * m + a);
      // symmetric: x - y = 0; skew-Hermitian: x + conj(y) = 0
      const double re = skew ? x[0] + y[0] : x[0] - y[0];
      const double im = skew ? x[1] - y[1] : x[1] - y[1];
      if (!(std::hypot(re, im) <= ND_INPUT_TOL * mx)) return false;
    }
  return true;
}

__global__ void k_check_H(const double* __restrict__ H, const int32_t* __restrict__ T, int nnz, double tol,
                          int* flag) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const double a = H[q], b = H[T[q]];
  if (!(fabs(a - b) <= tol * fmax(fabs(a), fabs(b)))) atomicOr(flag, 1);
}

// One CTA per (contact, energy): the largest magnitude of the block, then
// every pair (a, b), a <= b.
__global__ void k_check_blocks(const double2* __restrict__ S, int64_t stride, const int64_t* __restrict__ soff,
                               const int32_t* __restrict__ msz, int skew, double tol, int* flag) {
  const int c = blockIdx.x, e = blockIdx.y, m = msz[c];
  const double2* B = S + int64_t(e) * stride + soff[c];
  const int64_t mm = int64_t(m) * m;
  double mx = 0.0;
  bool bad = false;
  for (int64_t q = threadIdx.x; q < mm; q += blockDim.x) {
    const double a = hypot(B[q].x, B[q].y);
    if (!isfinite(a)) bad = true;
    mx = fmax(mx, a);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  for (int64_t q = threadIdx.x; q < mm && !bad; q += blockDim.x) {
    const int a = int(q / m), b = int(q % m);
    if (b < a) continue;
    const double2 x = B[q], y = B[int64_t(b) * m + a];
    const double re = skew ? x.x + y.x : x.x - y.x;
    const double im = skew ? x.y - y.y : x.y - y.y;
    if (!(hypot(re, im) <= tol * mx)) bad = true;
  }
  if (bad) atomicOr(flag, 1);
}

__global__ void k_check_diag_skew(const double2* __restrict__ s, int64_t count, double tol, int* flag) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const double2 v = s[q];
  if (!(fabs(v.x) <= tol * hypot(v.x, v.y))) atomicOr(flag, 1);
}

}  // namespace

nd_status host_check_factor(const nd_plan* p, const double* H, const double* sr, int n_e) {
  if (H) {
    const int32_t* T = csr_transpose(p);
    for (int q = 0; q < p->nnz; ++q) {
      const double a = H[q], b = H[T[q]];
      if (!close_sym(a, b, std::max(std::fabs(a), std::fabs(b))))
        return fail(ND_ERR_NOT_SYMMETRIC, "H values not symmetric (or not finite) at CSR entry " + std::to_string(q));
    }
  }
  if (sr)
    for (int e = 0; e < n_e; ++e)
      for (int c = 0; c < p->n_contacts; ++c) {
        const int m = p->contact_ptr[c + 1] - p->contact_ptr[c];
        if (!host_block_ok(sr + 2 * (int64_t(e) * p->sigma_elems + p->contact_soff[c]), m, false))
          return fail(ND_ERR_NOT_SYMMETRIC, "Sigma^r block of contact " + std::to_string(c) + " at energy " +
                                                std::to_string(e) + " not complex symmetric (or not finite)");
      }
  return ND_OK;
}

nd_status host_check_lesser(const nd_plan* p, const double* const blocks[2], const double* const diags[2], int n_e) {
  static const char* name[2] = {"Sigma^<", "Sigma^>"};
  for (int s = 0; s < 2; ++s) {
    if (blocks[s])
      for (int e = 0; e < n_e; ++e)
        for (int c = 0; c < p->n_contacts; ++c) {
          const int m = p->contact_ptr[c + 1] - p->contact_ptr[c];
          if (!host_block_ok(blocks[s] + 2 * (int64_t(e) * p->sigma_elems + p->contact_soff[c]), m, true))
            return fail(ND_ERR_NOT_SKEW_HERMITIAN, std::string(name[s]) + " block of contact " + std::to_string(c) +
                                                       " at energy " + std::to_string(e) +
                                                       " not skew-Hermitian (or not finite)");
        }
    if (diags[s])
      for (int64_t q = 0; q < int64_t(n_e) * p->n; ++q) {
        const double re = diags[s][2 * q], im = diags[s][2 * q + 1];
        if (!(std::fabs(re) <= ND_INPUT_TOL * std::hypot(re, im)))
          return fail(ND_ERR_NOT_SKEW_HERMITIAN, std::string("phonon ") + name[s] + " entry " + std::to_string(q) +
                                                     " has a real part (or is not finite)");
      }
  }
  return ND_OK;
}

void launch_check_H(const double* H, const int32_t* T, int nnz, int* flag, cudaStream_t s) {
  if (nnz > 0) k_check_H<<<(nnz + 255) / 256, 256, 0, s>>>(H, T, nnz, ND_INPUT_TOL, flag);
}

void launch_check_blocks(const double* S, int64_t stride, const int64_t* soff, const int32_t* m, int n_contacts,
                         int n_e, bool skew, int* flag, cudaStream_t s) {
  if (n_contacts > 0 && n_e > 0)
    k_check_blocks<<<dim3(n_contacts, n_e), 256, 0, s>>>(reinterpret_cast<const double2*>(S), stride, soff, m,
                                                         skew ? 1 : 0, ND_INPUT_TOL, flag);
}

void launch_check_diag_skew(const double* d, int64_t count, int* flag, cudaStream_t s) {
  if (count > 0)
    k_check_diag_skew<<<unsigned((count + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(d), count,
                                                                    ND_INPUT_TOL, flag);
}

}  // namespace ndgf

using namespace ndgf;

extern "C" nd_status nd_check_factor_inputs(const nd_plan* plan, const double* H_values, const double* sigma_r,
                                            int32_t n_e) {
  if (!plan || !H_values || n_e < 0) return fail(ND_ERR_INVALID_ARG, "nd_check_factor_inputs: bad argument");
  if (plan->n_contacts > 0 && n_e > 0 && !sigma_r)
    return fail(ND_ERR_INVALID_ARG, "nd_check_factor_inputs: sigma_r is NULL");
  return host_check_factor(plan, H_values, plan->n_contacts > 0 ? sigma_r : nullptr, n_e);
}

extern "C" nd_status nd_check_lesser_inputs(const nd_plan* plan, const double* sigma_lesser,
                                            const double* sigma_greater, const double* ph_lesser,
                                            const double* ph_greater, int32_t n_e) {
  if (!plan || n_e < 0) return fail(ND_ERR_INVALID_ARG, "nd_check_lesser_inputs: bad argument");
  const double* blocks[2] = {plan->n_contacts > 0 ? sigma_lesser : nullptr,
                             plan->n_contacts > 0 ? sigma_greater : nullptr};
  const double* diags[2] = {ph_lesser, ph_greater};
  return host_check_lesser(plan, blocks, diags, n_e);
}
