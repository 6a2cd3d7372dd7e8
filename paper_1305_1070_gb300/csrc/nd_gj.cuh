// Batched Gauss-Jordan inversion with partial pivoting, one CTA per matrix
// (device routine shared by the translation units that invert blocks).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "nd_arith.cuh"

namespace ndgf {

template <typename T> using O = Ops<T>;

// The elements start, start + step, ... of a row-major index space with
// `cols` columns, as (row, column) pairs updated without a division per
// element (callers keep rows * cols below 2^31).
struct Walk2 {
  int r, c, dr, dc, cols;
  __device__ __forceinline__ Walk2(int start, int step, int cols_) : cols(cols_) {
    r = start / cols;
    c = start - r * cols;
    dr = step / cols;
    dc = step - dr * cols;
  }
  __device__ __forceinline__ void next() {
    r += dr;
    c += dc;
    if (c >= cols) {
      c -= cols;
      ++r;
    }
  }
};

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

// Same inversion with two barriers per pivot step (gj_invert needs five):
//  A: with the pivot row p of column k known, R = (row p) / pivot (R_k =
//     1/pivot), the old row k moves to row p, colk = column k (row p's entry
//     read from the old row k);
//  B: every row i != k gets M_i -= colk_i R (column k starting from 0), row k
//     becomes R; the entries of column k+1 below row k compete for the next
//     pivot through an atomic maximum of (|x|^2 as float bits, -row) in
//     shared memory (largest magnitude, smallest row on ties).
// The column swaps of the pivoting are undone at the end by one gather per
// row.  Updates use Ops::sub_mul, which leaves FP32-pair entries unnormalised
// until they are next used as factors.  row and piv hold n ints, colk n
// elements, R n elements (all shared memory).
__device__ __forceinline__ unsigned long long gj_key(float mag, int i) {
  if (!(mag == mag)) mag = 0.f;  // NaN never wins
  return (static_cast<unsigned long long>(__float_as_uint(mag)) << 32) | static_cast<unsigned>(0x7fffffff - i);
}

template <typename TC>
__device__ void gj_invert2(cx<TC>* M, int n, int ld, int* piv, cx<TC>* colk, cx<TC>* R, int* n_singular) {
  // two key slots: step k reads slot k & 1 while its phase A clears the other
  __shared__ unsigned long long s_key[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_key[0] = s_key[1] = 0ull;
  __syncthreads();
  for (int i = tid; i < n; i += nt) atomicMax(&s_key[0], gj_key(float(O<TC>::mag2(M[int64_t(i) * ld])), i));
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int p = 0x7fffffff - int(unsigned(s_key[k & 1] & 0xffffffffull));
    cx<TC> pivot = O<TC>::norm(M[int64_t(p) * ld + k]);
    if (!(O<TC>::mag2(pivot) > typename O<TC>::R(0))) {  // exactly singular (or NaN): record, keep going
      if (tid == 0) atomicAdd(n_singular, 1);
      pivot = O<TC>::from_d2(make_double2(std::is_same<TC, double>::value ? 1e-300 : 1e-30, 0.0));
    }
    const cx<TC> inv = O<TC>::recip(pivot);
    // phase A: column k itself is not written here, so every thread reads the
    // pivot and column k unchanged; row p's entries are read by their own thread
    for (int j = tid; j < n; j += nt) {
      if (j == k) {
        R[j] = inv;
      } else {
        const cx<TC> a = O<TC>::norm(M[int64_t(p) * ld + j]);
        const cx<TC> b = M[int64_t(k) * ld + j];
        R[j] = O<TC>::mul(a, inv);
        if (p != k) M[int64_t(p) * ld + j] = b;
      }
      colk[j] = (j == k) ? O<TC>::zero() : O<TC>::norm(M[int64_t(j == p ? k : j) * ld + k]);
    }
    if (tid == 0) {
      piv[k] = p;
      s_key[(k + 1) & 1] = 0ull;
    }
    __syncthreads();
    const int nn = n * n;
    Walk2 wk(tid, nt, n);
    for (int idx = tid; idx < nn; idx += nt, wk.next()) {
      const int i = wk.r, j = wk.c;
      cx<TC>& a = M[int64_t(i) * ld + j];
      if (i == k) {
        a = R[j];
      } else {
        cx<TC> v = (j == k) ? O<TC>::zero() : a;
        O<TC>::sub_mul(v, colk[i], R[j]);
        a = v;
        if (j == k + 1 && i > k) atomicMax(&s_key[(k + 1) & 1], gj_key(float(O<TC>::mag2(v)), i));
      }
    }
    __syncthreads();
  }
  // Undo the column swaps: column j of the result is the current column
  // src[j], src = identity with the swaps (k, piv[k]) applied for k = n-1..0.
  // colk holds src (n ints fit in n elements), R the cycle-leader flags.
  int* src = reinterpret_cast<int*>(colk);
  int* lead = reinterpret_cast<int*>(R);
  if (tid == 0) {
    for (int j = 0; j < n; ++j) {
      src[j] = j;
      lead[j] = 0;
    }
    for (int k = n - 1; k >= 0; --k) {
      const int q = piv[k], t = src[k];
      src[k] = src[q];
      src[q] = t;
    }
    // mark the smallest index of every cycle of length > 1 (piv reused as visited flags)
    for (int j = 0; j < n; ++j) piv[j] = 0;
    for (int j = 0; j < n; ++j) {
      if (piv[j] || src[j] == j) continue;
      lead[j] = 1;
      for (int c = j; !piv[c]; c = src[c]) piv[c] = 1;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {  // in place along each cycle: new[j] = old[src[j]]
    cx<TC>* row = M + int64_t(i) * ld;
    for (int j0 = 0; j0 < n; ++j0) {
      if (!lead[j0]) continue;
      const cx<TC> t = row[j0];
      int j = j0;
      while (src[j] != j0) {
        row[j] = row[src[j]];
        j = src[j];
      }
      row[j] = t;
    }
    for (int j = 0; j < n; ++j) row[j] = O<TC>::norm(row[j]);
  }
  __syncthreads();
}

}  // namespace ndgf
