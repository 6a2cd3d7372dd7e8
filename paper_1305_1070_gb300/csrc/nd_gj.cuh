// Batched Gauss-Jordan inversion with partial pivoting, one CTA per matrix
// (device routine shared by the translation units that invert blocks).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "nd_arith.cuh"

namespace ndgf {

template <typename T> using O = Ops<T>;

// Batched in-place Gauss-Jordan inversion with partial pivoting (one CTA per
// matrix).  The matrix is n x n with leading dimension ld.
template <typename TC>
__device__ void gj_invert(cx<TC>* M, int n, int ld, int* piv, cx<TC>* colk, int* n_singular) {
  using R = typename O<TC>::R;
  __shared__ R red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
  for (int k = 0; k < n; ++k) {
    // pivot: largest |a_ik|^2 over i >= k (smallest index on ties)
    R bv = R(-1);
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const R v = O<TC>::mag2(M[int64_t(i) * ld + k]);
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      R v = red_v[0];
      int p = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < p)) {
          v = red_v[w];
          p = red_i[w];
        }
      s_p = p;
      piv[k] = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int j = tid; j < n; j += nt) {
        const cx<TC> t = M[int64_t(k) * ld + j];
        M[int64_t(k) * ld + j] = M[int64_t(p) * ld + j];
        M[int64_t(p) * ld + j] = t;
      }
    __syncthreads();
    cx<TC> pivot = M[int64_t(k) * ld + k];
    if (!(O<TC>::mag2(pivot) > R(0))) {  // exactly singular (or NaN): record, keep going
      if (tid == 0) atomicAdd(n_singular, 1);
      pivot = O<TC>::from_d2(make_double2(std::is_same<TC, double>::value ? 1e-300 : 1e-30, 0.0));
    }
    const cx<TC> inv = O<TC>::recip(pivot);
    for (int i = tid; i < n; i += nt) colk[i] = (i == k) ? O<TC>::zero() : M[int64_t(i) * ld + k];
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      cx<TC>& a = M[int64_t(k) * ld + j];
      a = (j == k) ? inv : O<TC>::mul(a, inv);
    }
    __syncthreads();
    const int64_t nn = int64_t(n) * n;
    for (int64_t idx = tid; idx < nn; idx += nt) {
      const int i = int(idx / n), j = int(idx % n);
      if (i == k) continue;
      cx<TC>& a = M[int64_t(i) * ld + j];
      const cx<TC> v = (j == k) ? O<TC>::zero() : a;
      a = O<TC>::sub(v, O<TC>::mul(colk[i], M[int64_t(k) * ld + j]));
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) {
        const cx<TC> t = M[int64_t(i) * ld + k];
        M[int64_t(i) * ld + k] = M[int64_t(i) * ld + p];
        M[int64_t(i) * ld + p] = t;
      }
    __syncthreads();
  }
}

}  // namespace ndgf
