// Device kernels of the nested-dissection NEGF path (sm_103a).
//
// Every kernel is batched over (descriptor, energy): blockIdx.x selects a
// descriptor (or a GEMM tile), blockIdx.y the energy.  Storage type T is
// double (complex128 path) or float (complex64 mixed path); complex numbers
// are interleaved double2 / float2.

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include <cstdint>

#include <type_traits>

#include "nd_arith.cuh"
#include "nd_gj.cuh"
#include "nd_kernels.h"

namespace ndgf {

// alpha and beta of an epilogue as a mode, decided once per CTA (the FP64
// compares would otherwise run per output on the slow FP64 pipe): 0 = the
// first special value (alpha 1, beta 0), 1 = the second (alpha -1, beta 1),
// 2 = general.
__host__ __device__ inline int scale_mode(double v, double first, double second) {
  return v == first ? 0 : (v == second ? 1 : 2);
}
// C = alpha P + beta D for the modes above (alpha: 0 keep, 1 negate; beta: 0
// none, 1 add D)
template <typename T>
__device__ __forceinline__ cx<T> epilogue(cx<T> r, int amode, double alpha, int bmode, double beta,
                                          const cx<T>* __restrict__ D, int64_t at) {
  if (amode == 1)
    r = O<T>::neg(r);
  else if (amode == 2)
    r = O<T>::scale(r, alpha);
  if (bmode) {
    const cx<T> dv = D[at];
    r = O<T>::add(r, bmode == 1 ? dv : O<T>::scale(dv, beta));
  }
  return r;
}

__device__ __forceinline__ double fermi_dev(double E, double mu, double kT) {
  double x = (E - mu) / kT;
  if (x > 0) {
    double ex = exp(-x);
    return ex / (1.0 + ex);
  }
  return 1.0 / (1.0 + exp(x));
}

// ---------------------------------------------------------------------------
// S1 assembly: F = [A_ii | A_iB] with A = (E + i eta) I - H - Sigma; BB = 0.
template <typename T>
__global__ void k_assemble(const AssembleDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                           const int32_t* __restrict__ ent_dst, const int32_t* __restrict__ ent_src,
                           const int32_t* __restrict__ sites, const double* __restrict__ H,
                           const double* __restrict__ energies, double eta, const double2* __restrict__ sigma_r,
                           int64_t sigma_stride, const double2* __restrict__ ph_r, int n, DelayTabs dt) {
  const AssembleDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* F = arena + int64_t(e) * se + d.off_F;
  cx<T>* BB = arena + int64_t(e) * se + d.off_BB;
  const int64_t nf = int64_t(d.n) * d.ld, nb = int64_t(d.b) * d.b;
  for (int64_t i = threadIdx.x; i < nf; i += blockDim.x) F[i] = O<T>::zero();
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) BB[i] = O<T>::zero();
  __syncthreads();
  for (int i = d.ent_begin + threadIdx.x; i < d.ent_end; i += blockDim.x)
    F[ent_dst[i]] = O<T>::from_d2(make_double2(-H[ent_src[i]], 0.0));
  __syncthreads();
  if (dt.iperm) {  // static row order and sites; virtual rows get their site from the child
    for (int r = threadIdx.x; r < d.n; r += blockDim.x) dt.iperm[int64_t(e) * dt.n_unk + d.site_begin + r] = r;
    for (int r = threadIdx.x; r < d.n_own; r += blockDim.x)
      dt.rsite[int64_t(e) * dt.n_unk + d.site_begin + r] = sites[d.site_begin + r];
  }
  const double E = energies[e];
  for (int r = threadIdx.x; r < d.n_own; r += blockDim.x) {
    double2 z = make_double2(E, eta);
    if (ph_r) {
      const double2 p = ph_r[int64_t(e) * n + sites[d.site_begin + r]];
      z.x -= p.x;
      z.y -= p.y;
    }
    cx<T>& a = F[int64_t(r) * d.ld + r];
    const double2 av = O<T>::to_d2(a);
    a = O<T>::from_d2(make_double2(av.x + z.x, av.y + z.y));
  }
  __syncthreads();  // the contact blocks below update the same diagonal entries
  const double2* S = sigma_r + int64_t(e) * sigma_stride;
  for (int c = 0; c < 2; ++c) {
    const int r0 = c ? d.c1 : d.c0, m = c ? d.m1 : d.m0, so = c ? d.soff1 : d.soff0;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
      const int a = i / m, b = i % m;
      const double2 sv = S[so + i];
      cx<T>& f = F[int64_t(r0 + a) * d.ld + r0 + b];
      const double2 fv = O<T>::to_d2(f);
      f = O<T>::from_d2(make_double2(fv.x - sv.x, fv.y - sv.y));
    }
  }
}

template <typename T>
__global__ void k_inverse(const InvDesc* __restrict__ descs, cx<T>* arena, int64_t se, double2* scratch,
                          int64_t scratch_stride, int* n_singular, int smem_max_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const InvDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* M = arena + int64_t(e) * se + d.off;
  // shared memory: piv (n ints), colk and R (n elements of up to 16 bytes
  // each), then the block itself when it fits
  int* piv = reinterpret_cast<int*>(smem);
  const size_t colk_off = (size_t(d.n) * sizeof(int) + 15) & ~size_t(15);
  const size_t r_off = colk_off + size_t(d.n) * sizeof(double2);
  const int nn = d.n * d.n;  // n <= 8192 + delays (nd_fact_create): 32-bit indices
  if (!std::is_same<T, double>::value && d.fp64 && scratch) {  // root block in complex128
    double2* W = scratch + int64_t(e) * scratch_stride + d.scr;
    {
      Walk2 wk(threadIdx.x, blockDim.x, d.n);
      for (int i = threadIdx.x; i < nn; i += blockDim.x, wk.next()) W[i] = O<T>::to_d2(M[int64_t(wk.r) * d.ld + wk.c]);
    }
    __syncthreads();
    gj_invert2<double>(W, d.n, d.n, piv, reinterpret_cast<double2*>(smem + colk_off),
                       reinterpret_cast<double2*>(smem + r_off), n_singular);
    Walk2 wk(threadIdx.x, blockDim.x, d.n);
    for (int i = threadIdx.x; i < nn; i += blockDim.x, wk.next()) M[int64_t(wk.r) * d.ld + wk.c] = O<T>::from_d2(W[i]);
  } else if (d.n <= smem_max_n) {  // whole block resident in shared memory
    cx<T>* colk = reinterpret_cast<cx<T>*>(smem + colk_off);
    cx<T>* R = reinterpret_cast<cx<T>*>(smem + r_off);
    cx<T>* S = reinterpret_cast<cx<T>*>(smem + r_off + size_t(d.n) * sizeof(double2));
    {
      Walk2 wk(threadIdx.x, blockDim.x, d.n);
      for (int i = threadIdx.x; i < nn; i += blockDim.x, wk.next()) S[i] = M[int64_t(wk.r) * d.ld + wk.c];
    }
    __syncthreads();
    gj_invert2<T>(S, d.n, d.n, piv, colk, R, n_singular);
    Walk2 wk(threadIdx.x, blockDim.x, d.n);
    for (int i = threadIdx.x; i < nn; i += blockDim.x, wk.next()) M[int64_t(wk.r) * d.ld + wk.c] = S[i];
  } else {
    gj_invert2<T>(M, d.n, d.ld, piv, reinterpret_cast<cx<T>*>(smem + colk_off),
                  reinterpret_cast<cx<T>*>(smem + r_off), n_singular);
  }
}

// ---------------------------------------------------------------------------
// Batched complex GEMM, C = alpha op(A) op(B) + beta D, one CTA per BM x BN
// output tile.  Thread (tx, ty) owns rows ty + i*(BM/TM), columns
// tx + j*(BN/TN) of the tile.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(const GemmDesc* __restrict__ descs, const TileRef* __restrict__ tiles, cx<T>* arena, int64_t se,
       const cx<T>* __restrict__ aux, int64_t sa) {
  constexpr int NX = BN / TN, NY = BM / TM, NT = NX * NY;
  constexpr int LA = (BM * BK + NT - 1) / NT, LB = (BK * BN + NT - 1) / NT;  // staged loads per thread
  // two shared buffers: the next k-tile is fetched into registers while the
  // current one is used, then stored to the other buffer (one barrier per step)
  // staged tiles plus Re + Im of every element (3-multiplication products),
  // in dynamic shared memory (gemm_smem_bytes)
  using S = typename O<T>::S;
  extern __shared__ __align__(16) unsigned char gsm[];
  auto As = reinterpret_cast<cx<T>(*)[BK][BM + 1]>(gsm);
  auto Bs = reinterpret_cast<cx<T>(*)[BK][BN + 1]>(gsm + sizeof(cx<T>) * 2 * BK * (BM + 1));
  auto Ass = reinterpret_cast<S(*)[BK][BM + 1]>(gsm + sizeof(cx<T>) * 2 * BK * (BM + 1 + BN + 1));
  auto Bss = reinterpret_cast<S(*)[BK][BN + 1]>(gsm + sizeof(cx<T>) * 2 * BK * (BM + 1 + BN + 1) +
                                                sizeof(S) * 2 * BK * (BM + 1));
  const TileRef t = tiles[blockIdx.x];
  const GemmDesc d = descs[t.desc];
  const int64_t e = blockIdx.y;
  cx<T>* base = arena + e * se;
  const cx<T>* abase = aux + e * sa;
  const cx<T>* A = (d.offA & AUX_BIT) ? abase + (d.offA & ~AUX_BIT) : base + d.offA;
  const cx<T>* B = (d.offB & AUX_BIT) ? abase + (d.offB & ~AUX_BIT) : base + d.offB;
  const int m0 = t.tm * BM, n0 = t.tn * BN;
  const int tid = threadIdx.x, tx = tid % NX, ty = tid / NX;
  const bool conjB = (d.opB == OP_C || d.opB == OP_H);
  const bool transB = (d.opB == OP_T || d.opB == OP_H);
  const bool transA = (d.opA != OP_N);
  cx<T> ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + l * NT;
      cx<T> v = O<T>::zero();
      if (idx < BM * BK) {
        const int mm = transA ? idx % BM : idx / BK, kk = transA ? idx / BM : idx % BK;
        const int gm = m0 + mm, gk = k0 + kk;
        if (gm < d.m && gk < d.k) v = transA ? A[int64_t(gk) * d.lda + gm] : A[int64_t(gm) * d.lda + gk];
      }
      ra[l] = v;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + l * NT;
      cx<T> v = O<T>::zero();
      if (idx < BK * BN) {
        const int kk = transB ? idx % BK : idx / BN, nn = transB ? idx / BK : idx % BN;
        const int gk = k0 + kk, gn = n0 + nn;
        if (gk < d.k && gn < d.n) v = transB ? B[int64_t(gn) * d.ldb + gk] : B[int64_t(gk) * d.ldb + gn];
      }
      rb[l] = conjB ? O<T>::conj(v) : v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + l * NT;
      if (idx < BM * BK) {
        const int mm = transA ? idx % BM : idx / BK, kk = transA ? idx / BM : idx % BK;
        As[buf][kk][mm] = ra[l];
        Ass[buf][kk][mm] = O<T>::sum(ra[l]);
      }
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + l * NT;
      if (idx < BK * BN) {
        const int kk = transB ? idx % BK : idx / BN, nn = transB ? idx / BK : idx % BN;
        Bs[buf][kk][nn] = rb[l];
        Bss[buf][kk][nn] = O<T>::sum(rb[l]);
      }
    }
  };
  typename O<T>::Acc3 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = O<T>::acc3_zero();
  const int nk = (d.k + BK - 1) / BK;
  if (nk > 0) {
    fetch(0);
    store(0);
  }
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) fetch((kt + 1) * BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cx<T> a[TM], b[TN];
      S as[TM], bs[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        a[i] = As[cur][kk][ty + i * NY];
        as[i] = Ass[cur][kk][ty + i * NY];
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        b[j] = Bs[cur][kk][tx + j * NX];
        bs[j] = Bss[cur][kk][tx + j * NX];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) O<T>::acc3_fma(acc[i][j], a[i], as[i], b[j], bs[j]);
    }
    if (kt + 1 < nk) store(cur ^ 1);
    __syncthreads();
  }
  cx<T>* C = base + d.offC;
  const cx<T>* D = base + d.offD;
  const int amode = scale_mode(d.alpha, 1.0, -1.0), bmode = scale_mode(d.beta, 0.0, 1.0);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NY;
    if (gm >= d.m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NX;
      if (gn >= d.n) continue;
      C[int64_t(gm) * d.ldc + gn] = epilogue<T>(O<T>::acc3_get(acc[i][j]), amode, d.alpha, bmode, d.beta, D, int64_t(gm) * d.ldd + gn);
    }
  }
}

// GEMM of small blocks (edges up to 96): one CTA per descriptor and energy,
// each thread a 2 x 2 block of outputs (the two rows of A and two columns of B
// it loads serve four multiply-adds), operands read through L1 without
// staging (no tile padding, no barriers); four real products per
// multiply-add (the 3-multiplication sums would be formed per loaded term).
template <typename T>
__global__ void __launch_bounds__(128) k_gemm_direct(const GemmDesc* __restrict__ descs,
                                                     const TileRef* __restrict__ tiles, cx<T>* arena, int64_t se,
                                                     const cx<T>* __restrict__ aux, int64_t sa) {
  const GemmDesc d = descs[tiles[blockIdx.x].desc];
  const int64_t e = blockIdx.y;
  cx<T>* base = arena + e * se;
  const cx<T>* abase = aux + e * sa;
  const cx<T>* A = (d.offA & AUX_BIT) ? abase + (d.offA & ~AUX_BIT) : base + d.offA;
  const cx<T>* B = (d.offB & AUX_BIT) ? abase + (d.offB & ~AUX_BIT) : base + d.offB;
  cx<T>* C = base + d.offC;
  const cx<T>* D = base + d.offD;
  const bool transA = d.opA != OP_N;
  const bool conjB = (d.opB == OP_C || d.opB == OP_H);
  const bool transB = (d.opB == OP_T || d.opB == OP_H);
  const int mb = (d.m + 1) >> 1, nb = (d.n + 1) >> 1;
  const int64_t sAi = transA ? 1 : d.lda, sAk = transA ? d.lda : 1;  // A(i, k) = A[i sAi + k sAk]
  const int64_t sBj = transB ? d.ldb : 1, sBk = transB ? 1 : d.ldb;  // B(k, j) = B[k sBk + j sBj]
  const int amode = scale_mode(d.alpha, 1.0, -1.0), bmode = scale_mode(d.beta, 0.0, 1.0);
  for (int idx = threadIdx.x; idx < mb * nb; idx += blockDim.x) {
    const int i0 = 2 * (idx / nb), j0 = 2 * (idx % nb);
    const bool i1 = i0 + 1 < d.m, j1 = j0 + 1 < d.n;
    const cx<T>* a0p = A + i0 * sAi;
    const cx<T>* a1p = A + (i1 ? i0 + 1 : i0) * sAi;
    const cx<T>* b0p = B + j0 * sBj;
    const cx<T>* b1p = B + (j1 ? j0 + 1 : j0) * sBj;
    typename O<T>::Acc c00 = O<T>::acc_zero(), c01 = O<T>::acc_zero(), c10 = O<T>::acc_zero(),
                       c11 = O<T>::acc_zero();
    auto mac = [&](cx<T> a0, cx<T> a1, cx<T> b0, cx<T> b1) {
      if (conjB) {
        b0 = O<T>::conj(b0);
        b1 = O<T>::conj(b1);
      }
      O<T>::acc_fma(c00, a0, b0);
      O<T>::acc_fma(c01, a0, b1);
      O<T>::acc_fma(c10, a1, b0);
      O<T>::acc_fma(c11, a1, b1);
    };
    // two k per iteration: the eight loads of a pair are in flight together
    int k = 0;
    for (; k + 1 < d.k; k += 2) {
      const cx<T> a0 = a0p[0], a1 = a1p[0], b0 = b0p[0], b1 = b1p[0];
      const cx<T> a0n = a0p[sAk], a1n = a1p[sAk], b0n = b0p[sBk], b1n = b1p[sBk];
      a0p += 2 * sAk;
      a1p += 2 * sAk;
      b0p += 2 * sBk;
      b1p += 2 * sBk;
      mac(a0, a1, b0, b1);
      mac(a0n, a1n, b0n, b1n);
    }
    if (k < d.k) mac(a0p[0], a1p[0], b0p[0], b1p[0]);
    const typename O<T>::Acc* acc[4] = {&c00, &c01, &c10, &c11};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + (q >> 1), j = j0 + (q & 1);
      if ((q >> 1) && !i1) continue;
      if ((q & 1) && !j1) continue;
      C[int64_t(i) * d.ldc + j] = epilogue<T>(O<T>::acc_get(*acc[q]), amode, d.alpha, bmode, d.beta, D,
                                              int64_t(i) * d.ldd + j);
    }
  }
}

template <typename T>
void Kern<T>::gemm_direct(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, cudaStream_t s) {
  if (n_tiles <= 0 || w.n_e <= 0) return;
  k_gemm_direct<T><<<dim3(n_tiles, w.n_e), 128, 0, s>>>(d, tiles, (cx<T>*)w.arena, w.se, (const cx<T>*)w.aux, w.sa);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Delayed pivots (an extension of the paper's fold; paper Sec. 3.2 eliminates
// every interior row of a cluster at the cluster).  The k rows of the front
// that are handed to the parent are chosen on X = (interior block)^{-1},
// computed in complex64: repeatedly the row j with the largest |X_jj|, after
// which X is replaced by the inverse of the block without row and column j,
// X <- X - X[:, j] X[j, :] / X_jj.  A large X_jj means that eliminating the
// other rows first leaves a small pivot 1 / X_jj for row j, so the chosen rows
// are the near-singular directions of the block.  The front is then reordered
// (eliminated rows first, in their previous order, then the chosen rows), the
// per-energy row tables follow, and the chosen rows' own couplings
// [A_DD | A_DB] go to the boundary accumulator, whose first k rows and columns
// are the parent's virtual rows of this cluster.  One CTA per (cluster, energy).
template <typename T>
__global__ void k_delay(const DelayDesc* __restrict__ descs, cx<T>* arena, int64_t se, DelayTabs dt, int x_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_sel, s_nsing;
  const DelayDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  const int nf = d.nf, k = d.k, m = nf - k, ld = d.ld, bb = d.bb;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
  cx<T>* base = arena + int64_t(e) * se;
  cx<T>* F = base + d.off_F;
  cx<T>* BB = base + d.off_BB;
  cx<T>* S = base + d.off_S;
  const size_t o1 = (size_t(nf) * sizeof(int) + 15) & ~size_t(15);
  int* piv = reinterpret_cast<int*>(smem);
  float2* colk = reinterpret_cast<float2*>(smem + o1);
  int* perm = reinterpret_cast<int*>(smem + o1 + size_t(nf) * sizeof(float2));
  int* rs = perm + nf;
  int* alive = rs + nf;
  // nf x nf complex64 working inverse: in shared memory when the launch
  // reserved room for it (behind the index arrays and the row buffer R), else
  // in the nf x ld scratch
  const size_t oR = (o1 + size_t(nf) * sizeof(float2) + size_t(3) * nf * sizeof(int) + 15) & ~size_t(15);
  float2* Rrow = reinterpret_cast<float2*>(smem + oR);
  const size_t o2 = oR + size_t(nf) * sizeof(float2);
  float2* X = x_smem ? reinterpret_cast<float2*>(smem + o2) : reinterpret_cast<float2*>(S);
  const int nn = nf * nf;  // 32-bit indices (front sizes bounded by nd_fact_create)
  {
    Walk2 wk(tid, nt, nf);
    for (int i = tid; i < nn; i += nt, wk.next()) {
      const double2 v = O<T>::to_d2(F[int64_t(wk.r) * ld + wk.c]);
      X[i] = make_float2(float(v.x), float(v.y));
    }
  }
  for (int i = tid; i < nf; i += nt) alive[i] = 1;
  if (tid == 0) s_nsing = 0;
  __syncthreads();
  gj_invert2<float>(X, nf, nf, piv, colk, Rrow, &s_nsing);
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    float bv = -1.f;
    int bi = nf;
    for (int j = tid; j < nf; j += nt)
      if (alive[j]) {
        const float2 x = X[int64_t(j) * nf + j];
        const float v = x.x * x.x + x.y * x.y;
        if (v > bv) {  // j increases along a thread's loop: ties keep the smaller index
          bv = v;
          bi = j;
        }
      }
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_down_sync(0xffffffffu, bv, o);
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
      float v = red_v[0];
      int p = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < p)) {
          v = red_v[w];
          p = red_i[w];
        }
      if (p >= nf)  // no comparable value (NaN): take the first remaining row
        for (p = 0; p < nf && !alive[p]; ++p) {
        }
      s_sel = p;
      alive[p] = 0;
      perm[m + t] = p;
    }
    __syncthreads();
    const int j = s_sel;
    const float2 pj = X[int64_t(j) * nf + j];
    const float den = pj.x * pj.x + pj.y * pj.y;
    if (den > 0.f) {
      const float2 inv = make_float2(pj.x / den, -pj.y / den);
      Walk2 wk(tid, nt, nf);
      for (int i = tid; i < nn; i += nt, wk.next()) {
        const int a = wk.r, b = wk.c;
        if (!alive[a] || !alive[b]) continue;
        const float2 xa = X[int64_t(a) * nf + j], xb = X[int64_t(j) * nf + b];
        const float2 q = make_float2(xa.x * inv.x - xa.y * inv.y, xa.x * inv.y + xa.y * inv.x);
        X[i] = make_float2(X[i].x - (q.x * xb.x - q.y * xb.y), X[i].y - (q.x * xb.y + q.y * xb.x));
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    int q = 0;
    for (int j = 0; j < nf; ++j)
      if (alive[j]) perm[q++] = j;
  }
  __syncthreads();
  int32_t* ip = dt.iperm + int64_t(e) * dt.n_unk + d.sb;
  int32_t* rsite = dt.rsite + int64_t(e) * dt.n_unk + d.sb;
  for (int r = tid; r < nf; r += nt) {
    ip[perm[r]] = r;
    rs[r] = rsite[perm[r]];
  }
  __syncthreads();
  for (int r = tid; r < nf; r += nt) rsite[r] = rs[r];
  for (int j = tid; j < k; j += nt) dt.rsite[int64_t(e) * dt.n_unk + d.sb_p + d.dslot + j] = rs[m + j];
  const int nfl = nf * ld;
  {
    Walk2 wk(tid, nt, ld);
    for (int i = tid; i < nfl; i += nt, wk.next()) S[i] = F[int64_t(perm[wk.r]) * ld + (wk.c < nf ? perm[wk.c] : wk.c)];
  }
  __syncthreads();
  for (int i = tid; i < nfl; i += nt) F[i] = S[i];
  __syncthreads();
  for (int i = tid; i < k * bb; i += nt) {
    const int a = i / bb, c = i % bb;
    BB[int64_t(a) * bb + c] = F[int64_t(m + a) * ld + m + c];
  }
  for (int i = tid; i < (bb - k) * k; i += nt) {
    const int a = i / k, c = i % k;
    BB[int64_t(k + a) * bb + c] = F[int64_t(m + c) * ld + m + k + a];
  }
}

// Final cluster and row of every front row of one cluster (top down: a
// delayed row takes the final position of the parent's virtual row).
__global__ void k_loc(const LocDesc* __restrict__ descs, DelayTabs dt) {
  const LocDesc d = descs[blockIdx.x];
  const int64_t eb = int64_t(blockIdx.y) * dt.n_unk;
  for (int s = threadIdx.x; s < d.nf; s += blockDim.x) {
    const int r = dt.iperm[eb + d.sb + s];
    int q = d.cluster, row = r;
    if (r >= d.n) {
      const int64_t u = eb + d.sb_p + d.dslot + (r - d.n);
      q = dt.locq[u];
      row = dt.locr[u];
    }
    dt.locq[eb + d.sb + s] = q;
    dt.locr[eb + d.sb + s] = row;
  }
}

void launch_loc(const LocDesc* d, int count, int n_e, const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || n_e <= 0) return;
  k_loc<<<dim3(count, n_e), 128, 0, s>>>(d, dt);
}


// Extend-add of a child's update into its parent's front.  Entries whose row
// is a boundary site of the parent and whose column is interior to it are
// dropped: the front stores [X_II | X_IB] and X_BB only.
template <typename T>
__global__ void k_scatter(const ScatterDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                          const int32_t* __restrict__ maps) {
  const ScatterDesc d = descs[blockIdx.x];
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  const cx<T>* src = base + d.off_src;
  cx<T>* front = base + d.off_front;
  cx<T>* bb = base + d.off_bb;
  const int32_t* map = maps + d.map_begin;
  const int ldp = d.n_p + d.b_p, nfp = d.n_p + d.k_p;  // front rows of the parent: positions < nfp
  const int nb = d.b * d.b;  // b <= 32768 (nd_fact_create): 32-bit index arithmetic
  for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
    const int r = idx / d.b, s = idx - r * d.b;
    const int pr = map[r], ps = map[s];
    const cx<T> v = src[idx];
    if (pr < nfp) {
      cx<T>& f = front[int64_t(pr) * ldp + ps];
      f = O<T>::add(f, v);
    } else if (ps >= nfp) {
      cx<T>& f = bb[int64_t(pr - d.n_p) * d.b_p + (ps - d.n_p)];
      f = O<T>::add(f, v);
    }
  }
}

// Gather of X_BB for a child from the parent's [X_II | X_IB] and X_BB; the
// parent's X_BI is X_IB^T (G^r, complex symmetric) or -X_IB^dagger (G^<, G^>).
// With delayed pivots the parent's rows are in its per-energy order: a static
// front position is translated through the parent's iperm first.
template <typename T>
__global__ void k_gather(const GatherDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                         const int32_t* __restrict__ maps, int skew, DelayTabs dt) {
  const GatherDesc d = descs[blockIdx.x];
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  const int32_t* ip = dt.iperm ? dt.iperm + int64_t(blockIdx.y) * dt.n_unk + d.sb_p : nullptr;
  const int nfp = d.n_p + d.k_p;
  cx<T>* dst = base + d.off_dst;
  const cx<T>* front = base + d.off_front;
  const cx<T>* bb = base + d.off_bb;
  const int32_t* map = maps + d.map_begin;
  const int ldp = d.n_p + d.b_p;
  const int nb = d.b * d.b;  // b <= 32768 (nd_fact_create): 32-bit index arithmetic
  for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
    const int r = idx / d.b, s = idx - r * d.b;
    int pr = map[r], ps = map[s];
    if (ip) {
      if (pr < nfp) pr = ip[pr];
      if (ps < nfp) ps = ip[ps];
    }
    cx<T> v;
    if (pr < d.n_p) {
      v = front[int64_t(pr) * ldp + ps];
    } else if (ps < d.n_p) {
      v = front[int64_t(ps) * ldp + pr];
      if (skew) v = O<T>::neg(O<T>::conj(v));
    } else {
      v = bb[int64_t(pr - d.n_p) * d.b_p + (ps - d.n_p)];
    }
    dst[idx] = v;
  }
}

template <typename T>
__global__ void k_zero(const ZeroDesc* __restrict__ descs, cx<T>* arena, int64_t se) {
  const ZeroDesc d = descs[blockIdx.x];
  cx<T>* p = arena + int64_t(blockIdx.y) * se + d.off;
  const cx<T> z = O<T>::zero();
  for (int64_t i = threadIdx.x; i < d.count; i += blockDim.x) p[i] = z;
}

// N_{I,Y} = diag(Sigma_ph) conj([G_II | G_{I,anc}])  (paper Sec. 3.2, first G^< step)
template <typename T>
__global__ void k_nph(const NPhDesc* __restrict__ descs, cx<T>* arena, int64_t se, const int32_t* __restrict__ sites,
                      const double2* __restrict__ ph_l, const double2* __restrict__ ph_g, int n, DelayTabs dt) {
  const NPhDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* base = arena + int64_t(e) * se;
  cx<T>* N = base + d.off_NX;
  const cx<T>* G = base + d.off_G;
  const cx<T>* GX = base + d.off_GX;
  const double2* ph = (d.rhs ? ph_g : ph_l) + int64_t(e) * n;
  const int w = d.n + d.A;
  const int64_t tot = int64_t(d.n) * w;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / w), j = int(idx % w);
    const int site = dt.rsite ? dt.rsite[int64_t(e) * dt.n_unk + d.site_begin + r] : sites[d.site_begin + r];
    const double2 s = ph[site];
    const cx<T> g = j < d.n ? G[int64_t(r) * d.ldG + j] : GX[int64_t(r) * d.A + (j - d.n)];
    N[idx] = O<T>::mul(O<T>::from_d2(s), O<T>::conj(g));
  }
}

// G_{B_i, anc(i)} from the G_II and G_{I,anc} blocks of the ancestors: the
// entry between unknowns x and y is stored by the lower of the two clusters
// that eliminate them (G^r is complex symmetric); the column of an unknown
// eliminated as row p of cluster o inside the ancestor columns of cluster q
// is A_q - n_o - A_o + p.  Ancestor column j is row anc_r[j] of cluster
// anc_q[j]; a boundary unknown's cluster and row are static, or per energy
// with delayed pivots.
template <typename T>
__global__ void k_gather_anc(const AncGatherDesc* __restrict__ descs, cx<T>* arena, int64_t se, AncTables t,
                             DelayTabs dt) {
  const AncGatherDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* base = arena + int64_t(e) * se;
  cx<T>* dst = base + d.off_dst;
  const int64_t tot = int64_t(d.b) * d.A;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / d.A), j = int(idx % d.A);
    const int u = t.site_ids[d.bsite_begin + r];
    int qx, px;
    if (dt.locq) {
      qx = dt.locq[int64_t(e) * dt.n_unk + u];
      px = dt.locr[int64_t(e) * dt.n_unk + u];
    } else {
      qx = t.unk_q[u];
      px = t.unk_r[u];
    }
    const int qy = t.anc_q[d.anc_begin + j], py = t.anc_r[d.anc_begin + j];
    int64_t src;
    if (qx == qy)
      src = t.cl_offG[qx] + int64_t(px) * t.cl_ldG[qx] + py;
    else if (qx < qy)
      src = t.cl_offGX[qx] + int64_t(px) * t.cl_A[qx] + (t.cl_A[qx] - t.cl_n[qy] - t.cl_A[qy] + py);
    else
      src = t.cl_offGX[qy] + int64_t(py) * t.cl_A[qy] + (t.cl_A[qy] - t.cl_n[qx] - t.cl_A[qx] + px);
    dst[idx] = base[src];
  }
}

// Rows of a child's N fold update into its parent: rows of I_p go to the
// parent's N_{I_p, Y_p} (same columns), rows of B_p to its accumulator
// N_{B_p, anc(p)} (columns of I_p there are dead lower blocks and dropped).
template <typename T>
__global__ void k_scatter_rows(const RowScatterDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                               const int32_t* __restrict__ maps, DelayTabs dt) {
  const RowScatterDesc d = descs[blockIdx.x];
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  const int32_t* ip = dt.iperm ? dt.iperm + int64_t(blockIdx.y) * dt.n_unk + d.sb_p : nullptr;
  const int nfp = d.n_p + d.k_p;
  const cx<T>* src = base + d.off_src;
  cx<T>* nx = base + d.off_nx;
  cx<T>* nb = base + d.off_nb;
  const int32_t* map = maps + d.map_begin;
  const int64_t tot = int64_t(d.b) * d.A_c;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / d.A_c), j = int(idx % d.A_c);
    int pr = map[r];
    if (ip && pr < nfp) pr = ip[pr];
    const cx<T> v = src[idx];
    if (pr < d.n_p) {
      cx<T>& f = nx[int64_t(pr) * d.A_c + j];
      f = O<T>::add(f, v);
    } else if (j >= d.n_p) {
      cx<T>& f = nb[int64_t(pr - d.n_p) * d.A_p + (j - d.n_p)];
      f = O<T>::add(f, v);
    }
  }
}

// [P_II | P_IB] = columns I_i and B_i of A_ii^{-1} N_{I,Y}.
template <typename T>
__global__ void k_colgather(const ColGatherDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                            const int32_t* __restrict__ cmaps, AncTables t, DelayTabs dt) {
  const ColGatherDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* base = arena + int64_t(e) * se;
  cx<T>* P = base + d.off_P;
  const cx<T>* PX = base + d.off_PX;
  const int w = d.n + d.b, wx = d.n + d.A;
  const int64_t tot = int64_t(d.n) * w;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / w), j = int(idx % w);
    int col = j;
    if (j >= d.n) {
      if (dt.locq) {  // boundary unknown: eliminated as row p of ancestor q
        const int u = t.site_ids[d.bsite_begin + j - d.n];
        const int q = dt.locq[int64_t(e) * dt.n_unk + u], pq = dt.locr[int64_t(e) * dt.n_unk + u];
        col = d.n + d.A - t.cl_n[q] - t.cl_A[q] + pq;
      } else {
        col = cmaps[d.cmap_begin + j - d.n];
      }
    }
    P[idx] = PX[int64_t(r) * wx + col];
  }
}

template <typename T>
__global__ void k_diag_out(const DiagDesc* __restrict__ descs, const cx<T>* arena, int64_t se,
                           const int32_t* __restrict__ sites, double2* out, int n, DelayTabs dt) {
  const DiagDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  const cx<T>* X = arena + int64_t(e) * se + d.off;
  for (int r = threadIdx.x; r < d.n; r += blockDim.x) {
    const int site = dt.rsite ? dt.rsite[int64_t(e) * dt.n_unk + d.site_begin + r] : sites[d.site_begin + r];
    out[int64_t(e) * n + site] = O<T>::to_d2(X[int64_t(r) * d.ld + r]);
  }
}

template <typename T>
__global__ void k_convert_aux(const double2* __restrict__ lesser, const double2* __restrict__ greater, cx<T>* aux,
                              int64_t sigma_elems, int n_e) {
  const int64_t tot = int64_t(n_e) * sigma_elems;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < tot; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = i / sigma_elems, k = i % sigma_elems;
    const double2 l = lesser ? lesser[i] : make_double2(0.0, 0.0);
    const double2 g = greater ? greater[i] : make_double2(0.0, 0.0);
    aux[e * 2 * sigma_elems + k] = O<T>::from_d2(l);
    aux[e * 2 * sigma_elems + sigma_elems + k] = O<T>::from_d2(g);
  }
}

// ---------------------------------------------------------------------------
// S9 certificate: for every site j, in FP64 from the stored selected entries,
//   r_j  = sum_k A_jk G_kj - 1
//   r<_j = sum_k A_jk G<_kj - (Sigma^< G^a)_jj
// with A = (E + i eta - Sigma_ph) I - H - Sigma_contact.  Every nonzero A_jk
// pairs with a stored entry of G^(0) (paper Sec. 3.2: the stored entries
// cover the fill pattern): when j and k are eliminated by the same cluster,
// in its [X_II] block; otherwise in the [X_IB] block of the lower of the two
// clusters, at the boundary column of the other unknown.  With delayed pivots
// the eliminating cluster and row of every unknown are per energy (locq /
// locr), and the boundary column is that of the first slot on the unknown's
// path of delays that lies in a proper ancestor of the lower cluster.
// Per energy: max |r|, max |G_jj|, max |r<|, max |G<_jj|; entry 5 becomes 1
// when a stored entry was not found (a planner inconsistency, never expected);
// entries 6 and 7 are the residuals relative to the magnitude of their terms,
// max_j |r_j| / max_j (sum_k |A_jk| |G_kj|) and max_j |r<_j| / max_j
// (sum_k |A_jk| |G<_kj| + sum_k |Sigma^<_jk| |G_jk|): normwise backward errors
// of the diagonal entries, comparable with the unit roundoff of the arithmetic
// that produced G (normwise, because entries of G^< far below the largest
// ones can lie under the FP32 exponent range of the single-precision paths).
__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(__double_as_longlong(v)));
}

struct CertLoc {
  int q, r;
};

__device__ __forceinline__ CertLoc cert_loc(const CertArgs& a, const DelayTabs& dt, int64_t eb, int s) {
  if (dt.locq) return CertLoc{dt.locq[eb + s], dt.locr[eb + s]};
  return CertLoc{a.unk_q[s], a.unk_r[s]};
}

// Boundary column, in cluster q, of the unknown that starts in slot s (q is
// below the cluster that eliminates it); -1 when not found.
__device__ int cert_bcol(const CertArgs& a, const DelayTabs& dt, int64_t eb, int s, int q) {
  for (int it = 0; it < 256; ++it) {
    const int c = a.unk_q[s];
    if (c > q && a.cl[c].first_desc <= q) {  // s lies in a proper ancestor of q: binary search of q's boundary
      int lo = a.cl[q].bs, hi = lo + a.cl[q].b;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a.bslot[mid] < s)
          lo = mid + 1;
        else
          hi = mid;
      }
      return (lo < a.cl[q].bs + a.cl[q].b && a.bslot[lo] == s) ? a.bidx[lo] : -1;
    }
    const int rho = dt.iperm ? dt.iperm[eb + s] : a.unk_r[s];
    const int n = a.cl[c].n, par = a.cl[c].parent;
    if (rho < n || par < 0) return -1;  // eliminated at or below q: not an ancestor's unknown
    s = a.cl[par].sb + a.cl[c].dslot + (rho - n);
  }
  return -1;
}

// Where the entry X_xy of the unknowns in slots ux, uy (coupled, or the same)
// is stored: the cluster q whose front holds it, the element offset within
// that cluster's [X_II | X_IB] front, and whether the stored element is X_yx
// (*transposed).  Returns false when it is not stored.
__device__ bool cert_entry(const CertArgs& a, const DelayTabs& dt, int64_t eb, int ux, int uy, int* q, int64_t* idx,
                           bool* transposed) {
  const CertLoc lx = cert_loc(a, dt, eb, ux), ly = cert_loc(a, dt, eb, uy);
  if (lx.q == ly.q) {
    *q = lx.q;
    *idx = int64_t(lx.r) * a.cl[lx.q].ld + ly.r;
    *transposed = false;
    return true;
  }
  const bool x_low = lx.q < ly.q;  // the lower cluster (postorder) stores the pair in its I x B block
  const CertLoc lo = x_low ? lx : ly;
  const int b = cert_bcol(a, dt, eb, x_low ? uy : ux, lo.q);
  if (b < 0) return false;
  *q = lo.q;
  *idx = int64_t(lo.r) * a.cl[lo.q].ld + a.cl[lo.q].n + b;
  *transposed = !x_low;
  return true;
}

// |z| in FP32 for the magnitude sums of the backward errors (their
// normalisation needs a few digits; FP64 hypot per term would run on the
// slow FP64 pipe)
__device__ __forceinline__ double magf(double2 z) {
  const float x = float(z.x), y = float(z.y);
  return double(sqrtf(fmaf(x, x, y * y)));
}

template <typename T>
__global__ void k_certificate(CertArgs a, DelayTabs dt, const cx<T>* arena, int64_t se) {
  const int e = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const double2* ph_r = reinterpret_cast<const double2*>(a.ph_r);
  const double2* ph_l = reinterpret_cast<const double2*>(a.ph_l);
  const double2* sr = reinterpret_cast<const double2*>(a.sr);
  const double2* sl = reinterpret_cast<const double2*>(a.sl);
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool lost = false;
  if (j < a.n) {
    const cx<T>* base = arena + int64_t(e) * se;
    const int64_t eb = int64_t(e) * dt.n_unk;
    const int uj = a.slot[j];
    const CertLoc lj = cert_loc(a, dt, eb, uj);
    const CertCluster cj = a.cl[lj.q];
    const int64_t dj = int64_t(lj.r) * cj.ld + lj.r;
    const double2 gjj = O<T>::to_d2(base[cj.offG + dj]);
    double2 pjj = make_double2(0.0, 0.0);
    if (a.lesser) pjj = O<T>::to_d2(base[cj.offP + dj]);
    double2 d = make_double2(a.energies[e], a.eta);
    if (ph_r) {
      const double2 q = ph_r[int64_t(e) * a.n + j];
      d.x -= q.x;
      d.y -= q.y;
    }
    double2 rr = make_double2(d.x * gjj.x - d.y * gjj.y - 1.0, d.x * gjj.y + d.y * gjj.x);
    double2 rl = make_double2(d.x * pjj.x - d.y * pjj.y, d.x * pjj.y + d.y * pjj.x);
    double2 rhs = make_double2(0.0, 0.0);
    const double ad = magf(d);
    double sr_sum = ad * magf(gjj), sl_sum = ad * magf(pjj);  // magnitudes of the terms
    if (a.lesser && ph_l) {  // ph^<_j conj(G_jj)
      const double2 q = ph_l[int64_t(e) * a.n + j];
      rhs.x += q.x * gjj.x + q.y * gjj.y;
      rhs.y += q.y * gjj.x - q.x * gjj.y;
      sl_sum += magf(q) * magf(gjj);
    }
    for (int t = a.cptr[j]; t < a.cptr[j + 1]; ++t) {
      const int k = a.nb[t], src = a.coef[t];
      int q;
      int64_t idx;
      bool tr;  // stored element X_jk (tr = false) or X_kj (tr = true)
      if (!cert_entry(a, dt, eb, uj, a.slot[k], &q, &idx, &tr)) {
        lost = true;
        continue;
      }
      const double2 g = O<T>::to_d2(base[a.cl[q].offG + idx]);  // G_kj = G_jk (complex symmetric)
      double2 an;                                                // -A_jk
      if (src >= 0) {
        an = make_double2(a.H[src], 0.0);
      } else {
        an = sr[int64_t(e) * a.sstride + (-1 - src)];
        if (a.lesser && sl) {  // Sigma^<_jk conj(G_jk)
          const double2 q2 = sl[int64_t(e) * a.sstride + (-1 - src)];
          rhs.x += q2.x * g.x + q2.y * g.y;
          rhs.y += q2.y * g.x - q2.x * g.y;
          sl_sum += magf(q2) * magf(g);
        }
      }
      const double aa = magf(an);
      rr.x -= an.x * g.x - an.y * g.y;
      rr.y -= an.x * g.y + an.y * g.x;
      sr_sum += aa * magf(g);
      if (a.lesser) {
        double2 pv = O<T>::to_d2(base[a.cl[q].offP + idx]);
        if (!tr) pv = make_double2(-pv.x, pv.y);  // G<_kj = -conj(G<_jk)
        rl.x -= an.x * pv.x - an.y * pv.y;
        rl.y -= an.x * pv.y + an.y * pv.x;
        sl_sum += aa * magf(pv);
      }
    }
    rl.x -= rhs.x;
    rl.y -= rhs.y;
    v[0] = hypot(rr.x, rr.y);
    v[1] = hypot(gjj.x, gjj.y);
    v[2] = hypot(rl.x, rl.y);
    v[3] = hypot(pjj.x, pjj.y);
    v[4] = sr_sum;
    v[5] = sl_sum;
    for (int k = 0; k < 6; ++k)  // NaN -> +inf, so that the max reduction keeps it
      if (!(v[k] >= 0.0)) v[k] = __longlong_as_double(0x7ff0000000000000LL);
  }
  __shared__ double red[6][32];
  __shared__ int s_lost;
  if (threadIdx.x == 0) s_lost = 0;
  __syncthreads();
  if (lost) s_lost = 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) x = fmax(x, red[threadIdx.x][w]);
    atomic_max_pos(a.cert + int64_t(e) * 8 + (threadIdx.x < 4 ? threadIdx.x : threadIdx.x + 2), x);
  }
  if (threadIdx.x == 0 && s_lost) atomic_max_pos(a.cert + int64_t(e) * 8 + 5, 1.0);
}

// Growth indicator: out[e * 8 + 4] = max over the listed regions of max |x|.
// Largest |Re| or |Im| of an element, in FP32 (the leading part of an FP32
// pair): the growth indicator needs no more, and FP64 arithmetic here would
// run on the slow FP64 pipe.
__device__ __forceinline__ float mag_lead(const float4& v) { return fmaxf(fabsf(v.x), fabsf(v.z)); }
__device__ __forceinline__ float mag_lead(const float2& v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float mag_lead(const double2& v) { return float(fmax(fabs(v.x), fabs(v.y))); }

// Fold growth max |Psi| per energy: CTAs stride over the Psi blocks of all
// clusters (most are small), one atomic maximum per CTA.
template <typename T>
__global__ void __launch_bounds__(128) k_absmax(const ZeroDesc* __restrict__ descs, int n_desc, const cx<T>* arena,
                                                int64_t se, double* cert) {
  const int e = blockIdx.y;
  float m = 0.f;
  for (int c = blockIdx.x; c < n_desc; c += gridDim.x) {
    const ZeroDesc d = descs[c];
    const cx<T>* p = arena + int64_t(e) * se + d.off;
    for (int64_t i = threadIdx.x; i < d.count; i += blockDim.x) {
      const float a = mag_lead(p[i]);
      m = fmaxf(m, a == a ? a : __int_as_float(0x7f800000));  // NaN counts as infinite growth
    }
  }
  __shared__ float red[4];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomic_max_pos(cert + int64_t(e) * 8 + 4, double(m));
  }
}

// ---------------------------------------------------------------------------
// Host launch wrappers
// Large and small GEMM tiles per precision.  The FP64 pipe (and the FP32 pipe
// under the 48-operation FP32-pair multiply-add) is slow enough that one or
// four outputs per thread keep it busy; the small tile wastes less on the
// ragged 10-60 row blocks of the lower tree levels.
// Variant 0 large, 1 small, 2 extra large (64 x 64 tiles with 4 x 4 outputs
// per thread: a quarter of the shared-memory reads per multiply-add of the
// large tile, for the blocks of 64 and more rows; chosen by the tuner).
template <typename T, int V> struct GemmCfg;
template <> struct GemmCfg<double, 0> { static constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2; };
template <> struct GemmCfg<double, 1> { static constexpr int BM = 16, BN = 16, BK = 16, TM = 1, TN = 1; };
template <> struct GemmCfg<double, 2> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };
template <> struct GemmCfg<float, 0> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct GemmCfg<float, 1> { static constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2; };
template <> struct GemmCfg<float, 2> { static constexpr int BM = 128, BN = 64, BK = 8, TM = 8, TN = 4; };
template <> struct GemmCfg<DF, 0> { static constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2; };
template <> struct GemmCfg<DF, 1> { static constexpr int BM = 16, BN = 16, BK = 16, TM = 2, TN = 2; };
template <> struct GemmCfg<DF, 2> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };

template <typename T> int Kern<T>::gemm_tile(int variant) {
  return variant == 1 ? GemmCfg<T, 1>::BM : variant == 2 ? GemmCfg<T, 2>::BM : GemmCfg<T, 0>::BM;
}
template <typename T> int Kern<T>::gemm_tile_n(int variant) {
  return variant == 1 ? GemmCfg<T, 1>::BN : variant == 2 ? GemmCfg<T, 2>::BN : GemmCfg<T, 0>::BN;
}

template <typename T>
void Kern<T>::assemble(const Work& w, const AssembleDesc* d, int count, const int32_t* ent_dst, const int32_t* ent_src,
                       const int32_t* sites, const double* H, const double* energies, double eta,
                       const double* sigma_r, int64_t sigma_stride, const double* ph_r, int n,
                       const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_assemble<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, ent_dst, ent_src, sites, H, energies, eta,
                                                    (const double2*)sigma_r, sigma_stride, (const double2*)ph_r, n, dt);
}

template <typename T>
void Kern<T>::delay(const Work& w, const DelayDesc* d, int count, int max_nf, const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  const size_t base = ((((size_t(max_nf) * sizeof(int) + 15) & ~size_t(15)) + size_t(max_nf) * sizeof(float2) +
                        size_t(3) * max_nf * sizeof(int) + 15) & ~size_t(15)) +
                      size_t(max_nf) * sizeof(float2);
  const size_t xs = size_t(max_nf) * max_nf * sizeof(float2);
  const int x_smem = base + xs <= size_t(200 * 1024) ? 1 : 0;  // up to nf = 158
  const size_t shm = base + (x_smem ? xs : 0);
  const int nt = max_nf <= 12 ? 32 : max_nf <= 24 ? 64 : max_nf <= 48 ? 128 : max_nf <= 96 ? 256 : 512;
  k_delay<T><<<dim3(count, w.n_e), nt, shm, s>>>(d, (cx<T>*)w.arena, w.se, dt, x_smem);
}

template <typename T>
void Kern<T>::inverse(const Work& w, const InvDesc* d, int count, int max_n, double* scratch, int64_t scratch_stride,
                      int* n_singular, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  const size_t base = ((size_t(max_n) * sizeof(int) + 15) & ~size_t(15)) + size_t(2) * max_n * sizeof(double2);
  // blocks with base + n^2 elements within 200 KB (n <= 111 for 16-byte
  // elements) are inverted in shared memory; larger ones in place in global memory
  int cap = 0;
  while (base + size_t(cap + 1) * (cap + 1) * sizeof(cx<T>) <= size_t(200 * 1024)) ++cap;
  const int smem_max_n = cap < max_n ? cap : max_n;
  const size_t shm = base + size_t(smem_max_n) * smem_max_n * sizeof(cx<T>);
  // the n x n update of every pivot step is spread over the CTA: large blocks
  // (the few fronts near the root) get more threads
  const int nt = max_n <= 12 ? 32 : max_n <= 24 ? 64 : max_n <= 48 ? 128 : max_n <= 64 ? 256 : (max_n <= 128 ? 512 : 1024);
  k_inverse<T><<<dim3(count, w.n_e), nt, shm, s>>>(d, (cx<T>*)w.arena, w.se, (double2*)scratch, scratch_stride,
                                                   n_singular, smem_max_n);
}

template <typename T, int V>
static void launch_gemm(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, cudaStream_t s) {
  using G = GemmCfg<T, V>;
  constexpr int NT = (G::BM / G::TM) * (G::BN / G::TN);
  constexpr size_t shm = (sizeof(cx<T>) + sizeof(typename O<T>::S)) * 2 * G::BK * (G::BM + 1 + G::BN + 1);
  auto kern = k_gemm<T, G::BM, G::BN, G::BK, G::TM, G::TN>;
  kern<<<dim3(n_tiles, w.n_e), NT, shm, s>>>(d, tiles, (cx<T>*)w.arena, w.se, (const cx<T>*)w.aux, w.sa);
}

template <typename T>
void Kern<T>::gemm(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, int variant, cudaStream_t s) {
  if (n_tiles <= 0 || w.n_e <= 0) return;
  if (variant == 1)
    launch_gemm<T, 1>(w, d, tiles, n_tiles, s);
  else if (variant == 2)
    launch_gemm<T, 2>(w, d, tiles, n_tiles, s);
  else
    launch_gemm<T, 0>(w, d, tiles, n_tiles, s);
}

template <typename T>
void Kern<T>::scatter(const Work& w, const ScatterDesc* d, int count, const int32_t* maps, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_scatter<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, maps);
}

template <typename T>
void Kern<T>::gather(const Work& w, const GatherDesc* d, int count, const int32_t* maps, bool skew,
                     const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_gather<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, maps, skew ? 1 : 0, dt);
}

template <typename T>
void Kern<T>::zero(const Work& w, const ZeroDesc* d, int count, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_zero<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se);
}

template <typename T>
void Kern<T>::nph(const Work& w, const NPhDesc* d, int count, const int32_t* sites, const double* ph_l,
                  const double* ph_g, int n, const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_nph<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, sites, (const double2*)ph_l,
                                              (const double2*)ph_g, n, dt);
}

template <typename T>
void Kern<T>::gather_anc(const Work& w, const AncGatherDesc* d, int count, const AncTables& t, const DelayTabs& dt,
                         cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_gather_anc<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, t, dt);
}

template <typename T>
void Kern<T>::scatter_rows(const Work& w, const RowScatterDesc* d, int count, const int32_t* maps,
                           const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_scatter_rows<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, maps, dt);
}

template <typename T>
void Kern<T>::colgather(const Work& w, const ColGatherDesc* d, int count, const int32_t* cmaps, const AncTables& t,
                        const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_colgather<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, cmaps, t, dt);
}

template <typename T>
void Kern<T>::diag_out(const Work& w, const DiagDesc* d, int count, const int32_t* sites, double* out, int n,
                       const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_diag_out<T><<<dim3(count, w.n_e), 128, 0, s>>>(d, (const cx<T>*)w.arena, w.se, sites, (double2*)out, n, dt);
}

template <typename T>
void Kern<T>::convert_aux(const Work& w, const double* lesser, const double* greater, int64_t sigma_elems,
                          cudaStream_t s) {
  if (sigma_elems <= 0 || w.n_e <= 0) return;
  int64_t tot = int64_t(w.n_e) * sigma_elems;
  int blocks = int((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_convert_aux<T><<<blocks, 256, 0, s>>>((const double2*)lesser, (const double2*)greater, (cx<T>*)w.aux,
                                          sigma_elems, w.n_e);
}

// Selected entries G^r_xy, G^<_xy, G^>_xy of the pairs (x[p], y[p]) for every
// energy (out [n_e][count] complex; NaN and a count when not stored).
template <typename T>
__global__ void k_selected(CertArgs a, DelayTabs dt, const cx<T>* arena, int64_t se, const int32_t* __restrict__ px,
                           const int32_t* __restrict__ py, int count, int lesser, double2* Gr, double2* Gl,
                           double2* Gg, int* n_missing) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.y;
  if (p >= count) return;
  const cx<T>* base = arena + int64_t(e) * se;
  const int64_t eb = int64_t(e) * dt.n_unk, o = int64_t(e) * count + p;
  const int x = px[p], y = py[p];
  int q;
  int64_t idx;
  bool tr;
  if (x < 0 || y < 0 || x >= a.n || y >= a.n || !cert_entry(a, dt, eb, a.slot[x], a.slot[y], &q, &idx, &tr)) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (Gr) Gr[o] = make_double2(nan, nan);
    if (Gl) Gl[o] = make_double2(nan, nan);
    if (Gg) Gg[o] = make_double2(nan, nan);
    atomicAdd(n_missing, 1);
    return;
  }
  if (Gr) Gr[o] = O<T>::to_d2(base[a.cl[q].offG + idx]);
  if (lesser) {  // X_xy = -conj(X_yx) for the skew-Hermitian G^<, G^>
    double2 l = O<T>::to_d2(base[a.cl[q].offP + idx]), g = O<T>::to_d2(base[a.cl[q].offPg + idx]);
    if (tr) {
      l = make_double2(-l.x, l.y);
      g = make_double2(-g.x, g.y);
    }
    if (Gl) Gl[o] = l;
    if (Gg) Gg[o] = g;
  }
}

template <typename T>
void Kern<T>::selected(const Work& w, const CertArgs& a, const DelayTabs& dt, const int32_t* x, const int32_t* y,
                       int count, int lesser, double* Gr, double* Gl, double* Gg, int* n_missing, cudaStream_t s) {
  if (w.n_e <= 0 || count <= 0) return;
  k_selected<T><<<dim3((count + 255) / 256, w.n_e), 256, 0, s>>>(
      a, dt, (const cx<T>*)w.arena, w.se, x, y, count, lesser, (double2*)Gr, (double2*)Gl, (double2*)Gg, n_missing);
}

// Entries 6, 7 hold the largest term magnitudes after k_certificate: divide.
__global__ void k_cert_ratio(double* cert, int n_e) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  double* c = cert + int64_t(e) * 8;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  c[6] = c[6] > 0.0 ? c[0] / c[6] : (c[0] > 0.0 ? inf : 0.0);
  c[7] = c[7] > 0.0 ? c[2] / c[7] : (c[2] > 0.0 ? inf : 0.0);
}

template <typename T>
void Kern<T>::certificate(const Work& w, const CertArgs& a, const DelayTabs& dt, cudaStream_t s) {
  if (w.n_e <= 0) return;
  if (a.n_psi > 0)
    k_absmax<T><<<dim3(std::min(a.n_psi, 1024), w.n_e), 128, 0, s>>>(a.psi, a.n_psi, (const cx<T>*)w.arena, w.se,
                                                                    a.cert);
  k_certificate<T><<<dim3((a.n + 255) / 256, w.n_e), 256, 0, s>>>(a, dt, (const cx<T>*)w.arena, w.se);
  k_cert_ratio<<<(w.n_e + 127) / 128, 128, 0, s>>>(a.cert, w.n_e);
}

// S10 terminal current spectrum (Meir-Wingreen) of one contact:
//   i_c(E) = Tr[Sigma^<_c G^>_cc - Sigma^>_c G^<_cc]
// over the contact block, G^< and G^> from the contact cluster's [P_II | P_IB]
// fronts (rows row0 .. row0+m of its interior), Sigma from the FP64 inputs.
// One CTA per energy; out[e] = Re, out_im[e] = Im (zero up to rounding: the
// trace of a product of two skew-Hermitian matrices is real).
template <typename T>
__global__ void k_current(const cx<T>* arena, int64_t se, int64_t offPl, int64_t offPg, int ld, int row0, int m,
                          const double2* __restrict__ sl, const double2* __restrict__ sg, int64_t sstride, int64_t soff,
                          double* out, double* out_im) {
  const int e = blockIdx.x;
  const cx<T>* Pl = arena + int64_t(e) * se + offPl;
  const cx<T>* Pg = arena + int64_t(e) * se + offPg;
  const double2* L = sl + int64_t(e) * sstride + soff;
  const double2* Gt = sg + int64_t(e) * sstride + soff;
  double re = 0.0, im = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int a = idx / m, b = idx % m;
    const double2 s1 = L[idx], s2 = Gt[idx];
    const double2 gg = O<T>::to_d2(Pg[int64_t(row0 + b) * ld + row0 + a]);
    const double2 gl = O<T>::to_d2(Pl[int64_t(row0 + b) * ld + row0 + a]);
    re += (s1.x * gg.x - s1.y * gg.y) - (s2.x * gl.x - s2.y * gl.y);
    im += (s1.x * gg.y + s1.y * gg.x) - (s2.x * gl.y + s2.y * gl.x);
  }
  __shared__ double rr[32], ri[32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rr[threadIdx.x >> 5] = re;
    ri[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) {
      re += rr[w];
      im += ri[w];
    }
    out[e] = re;
    if (out_im) out_im[e] = im;
  }
}

template <typename T>
void Kern<T>::current(const Work& w, int64_t offPl, int64_t offPg, int ld, int row0, int m, const double* sl,
                      const double* sg, int64_t sstride, int64_t soff, double* out, double* out_im, cudaStream_t s) {
  if (w.n_e <= 0 || m <= 0) return;
  k_current<T><<<w.n_e, 256, 0, s>>>((const cx<T>*)w.arena, w.se, offPl, offPg, ld, row0, m, (const double2*)sl,
                                     (const double2*)sg, sstride, soff, out, out_im);
}

// ---------------------------------------------------------------------------
// Adjoint solves (nd_density_gradient): A X = R for M right-hand sides with
// the stored factorization, in the cluster layout of the fold.
//   upward:   RB_i += Psi_i^T XI_i, rows of RB_i added to the parent's XI / RB;
//   downward: XB_i gathered from the parent's XS / XB, XS_i = A_ii^{-1} XI_i + Psi_i XB_i.
template <typename T>
__global__ void k_rows_add(const RowsDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                           const int32_t* __restrict__ maps, int M, DelayTabs dt) {
  const RowsDesc d = descs[blockIdx.x];
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  const int32_t* ip = dt.iperm ? dt.iperm + int64_t(blockIdx.y) * dt.n_unk + d.sb_p : nullptr;
  const int32_t* map = maps + d.map_begin;
  const cx<T>* src = base + d.off_child;
  const int nfp = d.m_p + d.k_p;
  const int64_t tot = int64_t(d.b) * M;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / M), j = int(idx % M);
    int pr = map[r];
    if (ip && pr < nfp) pr = ip[pr];
    cx<T>& dst = pr < d.m_p ? base[d.off_pi + int64_t(pr) * M + j] : base[d.off_pb + int64_t(pr - d.m_p) * M + j];
    dst = O<T>::add(dst, src[idx]);
  }
}

template <typename T>
__global__ void k_rows_gather(const RowsDesc* __restrict__ descs, cx<T>* arena, int64_t se,
                              const int32_t* __restrict__ maps, int M, DelayTabs dt) {
  const RowsDesc d = descs[blockIdx.x];
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  const int32_t* ip = dt.iperm ? dt.iperm + int64_t(blockIdx.y) * dt.n_unk + d.sb_p : nullptr;
  const int32_t* map = maps + d.map_begin;
  cx<T>* dst = base + d.off_child;
  const int nfp = d.m_p + d.k_p;
  const int64_t tot = int64_t(d.b) * M;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / M), j = int(idx % M);
    int pr = map[r];
    if (ip && pr < nfp) pr = ip[pr];
    dst[idx] = pr < d.m_p ? base[d.off_pi + int64_t(pr) * M + j] : base[d.off_pb + int64_t(pr - d.m_p) * M + j];
  }
}

// Unit right-hand sides at the contact sites: element offsets (per energy) of
// the ones.
template <typename T>
__global__ void k_set_one(const int64_t* __restrict__ offs, int count, cx<T>* arena, int64_t se) {
  cx<T>* base = arena + int64_t(blockIdx.y) * se;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    base[offs[i]] = O<T>::from_d2(make_double2(1.0, 0.0));
}

// Between the two solves of one cluster (and RB = 0).
// Right-hand side of the second solve from the first one's solution U:
// diag(c) conj(U) (adjoint, mode bit 0 clear) or diag(c) U (forward, bit 0
// set); U is XS of the first solve, saved here (bit 1 clear), or the copy an
// earlier call saved (bit 1 set).
template <typename T>
__global__ void k_adj_mid(const AdjDesc* __restrict__ descs, cx<T>* arena, int64_t se, int M,
                          const double* __restrict__ c, const int32_t* __restrict__ sites, DelayTabs dt, int mode) {
  const AdjDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  cx<T>* base = arena + int64_t(e) * se;
  const int64_t tot = int64_t(d.m) * M;
  for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = int(idx / M);
    const int site = dt.rsite ? dt.rsite[int64_t(e) * dt.n_unk + d.site_begin + r] : sites[d.site_begin + r];
    cx<T> x;
    if (mode & 2) {
      x = base[d.off_U + idx];
    } else {
      x = base[d.off_XS + idx];
      base[d.off_U + idx] = x;
    }
    base[d.off_XI + idx] = O<T>::scale((mode & 1) ? x : O<T>::conj(x), c[site]);
  }
  const int64_t tb = int64_t(d.b) * M;
  for (int64_t idx = threadIdx.x; idx < tb; idx += blockDim.x) base[d.off_RB + idx] = O<T>::zero();
}

// Adjoint (forward = 0): t_k = sum_{a,b} Sigma^<_ab conj(U_kb) conj(Z_ka);
// forward (forward = 1): T_k = sum_{a,b} W_ka Sigma^<_ab conj(U_kb); over the
// contact blocks, for every eliminated row k of one cluster (Z or W = XS of
// the second solve); one warp per row, in complex128.
template <typename T>
__global__ void k_adj_contract(const AdjDesc* __restrict__ descs, const cx<T>* arena, int64_t se, int M,
                               ContactTable ct, const double2* __restrict__ sl, int64_t sstride,
                               const int32_t* __restrict__ sites, DelayTabs dt, double2* out, int n, int forward) {
  const AdjDesc d = descs[blockIdx.x];
  const int e = blockIdx.y;
  const cx<T>* base = arena + int64_t(e) * se;
  const double2* S = sl + int64_t(e) * sstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < d.m; r += nw) {
    const cx<T>* U = base + d.off_U + int64_t(r) * M;
    const cx<T>* Z = base + d.off_XS + int64_t(r) * M;
    double re = 0.0, im = 0.0;
    int col0 = 0;
    for (int c = 0; c < ct.n; ++c) {
      const int m = ct.m[c];
      const double2* Sc = S + ct.off[c];
      for (int a = lane; a < m; a += 32) {
        const double2 za = O<T>::to_d2(Z[col0 + a]);
        double sr = 0.0, si = 0.0;  // sum_b S_ab conj(U_b)
        for (int bb = 0; bb < m; ++bb) {
          const double2 s = Sc[int64_t(a) * m + bb];
          const double2 u = O<T>::to_d2(U[col0 + bb]);
          sr += s.x * u.x + s.y * u.y;
          si += s.y * u.x - s.x * u.y;
        }
        if (forward) {  // (sr + i si) za
          re += sr * za.x - si * za.y;
          im += si * za.x + sr * za.y;
        } else {  // (sr + i si) conj(za)
          re += sr * za.x + si * za.y;
          im += si * za.x - sr * za.y;
        }
      }
      col0 += m;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      const int site = dt.rsite ? dt.rsite[int64_t(e) * dt.n_unk + d.site_begin + r] : sites[d.site_begin + r];
      out[int64_t(e) * n + site] = make_double2(re, im);
    }
  }
}

template <typename T>
void Kern<T>::rows(const Work& w, const RowsDesc* d, int count, const int32_t* maps, int M, bool gather,
                   const DelayTabs& dt, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  if (gather)
    k_rows_gather<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, maps, M, dt);
  else
    k_rows_add<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, maps, M, dt);
}

template <typename T>
__global__ void k_zero_range(cx<T>* arena, int64_t se, int64_t off, int64_t count) {
  cx<T>* p = arena + int64_t(blockIdx.y) * se + off;
  const cx<T> z = O<T>::zero();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z;
}

template <typename T>
void Kern<T>::zero_range(const Work& w, int64_t off, int64_t count, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  int blocks = int(std::min<int64_t>((count + 255) / 256, 1024));
  k_zero_range<T><<<dim3(blocks, w.n_e), 256, 0, s>>>((cx<T>*)w.arena, w.se, off, count);
}

template <typename T>
void Kern<T>::adj_ones(const Work& w, const int64_t* offs, int count, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_set_one<T><<<dim3((count + 255) / 256, w.n_e), 256, 0, s>>>(offs, count, (cx<T>*)w.arena, w.se);
}

template <typename T>
void Kern<T>::adj_mid(const Work& w, const AdjDesc* d, int count, int M, const double* c, const int32_t* sites,
                      const DelayTabs& dt, int mode, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_adj_mid<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (cx<T>*)w.arena, w.se, M, c, sites, dt, mode);
}

template <typename T>
void Kern<T>::adj_contract(const Work& w, const AdjDesc* d, int count, int M, const ContactTable& ct,
                           const double* sl, int64_t sstride, const int32_t* sites, const DelayTabs& dt,
                           double* out, int n, int forward, cudaStream_t s) {
  if (count <= 0 || w.n_e <= 0) return;
  k_adj_contract<T><<<dim3(count, w.n_e), 256, 0, s>>>(d, (const cx<T>*)w.arena, w.se, M, ct, (const double2*)sl,
                                                       sstride, sites, dt, (double2*)out, n, forward);
}

// Dynamic shared memory limits of every kernel that may need more than 48 KB
// (k_delay and k_inverse up to ~200 KB, the large GEMM tiles, k_gemm_tc),
// set once per device, before any launch can be recorded into a graph.
// The largest dynamic shared memory a kernel may take: the device's opt-in
// limit per block less the kernel's static shared memory.
template <typename K>
static void allow_max_smem(K kern, int optin) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
}

template <typename T>
static void prepare_t(int optin) {
  allow_max_smem(k_delay<T>, optin);
  allow_max_smem(k_inverse<T>, optin);
  using GL = GemmCfg<T, 0>;
  using GS = GemmCfg<T, 1>;
  using GX = GemmCfg<T, 2>;
  allow_max_smem(k_gemm<T, GL::BM, GL::BN, GL::BK, GL::TM, GL::TN>, optin);
  allow_max_smem(k_gemm<T, GS::BM, GS::BN, GS::BK, GS::TM, GS::TN>, optin);
  allow_max_smem(k_gemm<T, GX::BM, GX::BN, GX::BK, GX::TM, GX::TN>, optin);
}

void prepare_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  int optin = 48 * 1024;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  prepare_t<double>(optin);
  prepare_t<float>(optin);
  prepare_t<DF>(optin);
  prepare_gemm_tc();
  cudaGetLastError();
  done[dev] = true;
}

template struct Kern<double>;
template struct Kern<float>;
template struct Kern<DF>;

// ---------------------------------------------------------------------------
// S10 density: out_j (+)= scale * sum_e w_e Im X[e][j]   (X = diag G^<, caller order)
__global__ void k_density(const double2* __restrict__ X, const double* __restrict__ w, int n_e, int n, double scale,
                          int accumulate, double* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = 0; e < n_e; ++e) acc = fma(w[e], X[int64_t(e) * n + j].y, acc);
    out[j] = (accumulate ? out[j] : 0.0) + scale * acc;
  }
}

void launch_density(const double* X, const double* w, int n_e, int n, double scale, int accumulate, double* out,
                    cudaStream_t s) {
  int blocks = (n + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_density<<<blocks, 256, 0, s>>>((const double2*)X, w, n_e, n, scale, accumulate, out);
}

// ---------------------------------------------------------------------------
// S1a contact self-energy of a lead with H01 = -h I, tau = -h I, in the
// transverse-mode basis H00 = U diag(eps) U^T (FP64 always).
__device__ __forceinline__ double2 csqrt_dev(double2 w) {
  double r = hypot(w.x, w.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  double a = sqrt(0.5 * (r + fabs(w.x)));
  if (w.x >= 0.0) return make_double2(a, w.y / (2.0 * a));
  return make_double2(fabs(w.y) / (2.0 * a), copysign(a, w.y));
}

__global__ void k_lead_modes(const double* __restrict__ U, const double* __restrict__ eps, int m, double hop,
                             const double* __restrict__ energies, double eta, double2* out, int64_t stride,
                             int64_t offset) {
  extern __shared__ double2 lam[];
  const int e = blockIdx.y;
  const double E = energies[e];
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    // lambda^2 - x lambda + 1 = 0, x = (z - eps)/h; keep the root with |lambda| < 1
    const double2 x = make_double2((E - eps[q]) / hop, eta / hop);
    const double2 w = make_double2(x.x * x.x - x.y * x.y - 4.0, 2.0 * x.x * x.y);
    const double2 rt = csqrt_dev(w);
    const double2 p = make_double2(x.x + rt.x, x.y + rt.y), mns = make_double2(x.x - rt.x, x.y - rt.y);
    const double2 big = (p.x * p.x + p.y * p.y >= mns.x * mns.x + mns.y * mns.y) ? p : mns;
    // lambda = 2 / big (product of the roots is 1)
    const double den = big.x * big.x + big.y * big.y;
    lam[q] = make_double2(hop * 2.0 * big.x / den, -hop * 2.0 * big.y / den);
  }
  __syncthreads();
  const int64_t mm = int64_t(m) * m;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < mm; idx += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(idx / m), k = int(idx % m);
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < m; ++q) {
      const double u = U[int64_t(j) * m + q] * U[int64_t(k) * m + q];
      sr = fma(u, lam[q].x, sr);
      si = fma(u, lam[q].y, si);
    }
    out[int64_t(e) * stride + offset + idx] = make_double2(sr, si);
  }
}

void launch_lead_modes(const double* U, const double* eps, int m, double hop, const double* energies, int n_e,
                       double eta, double* out, int64_t stride, int64_t offset, cudaStream_t s) {
  const int64_t mm = int64_t(m) * m;
  int bx = int((mm + 255) / 256);
  if (bx > 64) bx = 64;
  k_lead_modes<<<dim3(bx, n_e), 256, size_t(m) * sizeof(double2), s>>>(U, eps, m, hop, energies, eta, (double2*)out,
                                                                       stride, offset);
}

// ---------------------------------------------------------------------------
// S1a for a general lead: renormalisation-decimation of Lopez Sancho, Lopez
// Sancho and Rubio (J. Phys. F 15, 851 (1985)) in complex128, one CTA per
// energy.  Layers 1, 2, ... of the lead have on-site block H00 and hopping H01
// from a layer to the next; every step eliminates every other remaining layer,
// doubling the reach of the effective couplings a (outwards) and b (inwards):
//   g = (z - e)^{-1};  e_s += a g b;  e += a g b + b g a;  a <- a g a;  b <- b g b
// with e_s = e = H00, a = H01, b = H01^T at the start.  The loop ends when
// every |a_ij|, |b_ij| < tol * scale (scale = max(1, max|H00|, max|H01|)) or
// after max_iter steps (counted in status[0]); then g_s = (z - e_s)^{-1} and
// Sigma = tau g_s tau^T.  Singular pivots of the inversions go to status[1].

// C = A B, all m x m row major, CTA-wide; ends with a barrier.
__device__ void cta_matmul(double2* __restrict__ C, const double2* __restrict__ A, const double2* __restrict__ B,
                           int rows, int inner, int cols, bool transB) {
  for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
    const int i = idx / cols, j = idx % cols;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < inner; ++k) {
      const double2 a = A[i * inner + k], b = transB ? B[j * inner + k] : B[k * cols + j];
      re = fma(a.x, b.x, re);
      re = fma(-a.y, b.y, re);
      im = fma(a.x, b.y, im);
      im = fma(a.y, b.x, im);
    }
    C[idx] = make_double2(re, im);
  }
  __syncthreads();
}

__global__ void k_lead_decimation(const double* __restrict__ H00, const double* __restrict__ H01,
                                  const double* __restrict__ tau, int m, int m_c,
                                  const double* __restrict__ energies, double eta, double scale, double tol,
                                  int max_iter, double2* __restrict__ out, int64_t stride, int64_t offset,
                                  double2* __restrict__ work, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_big;
  const int e = blockIdx.x;
  const int mm = m * m, mx = m_c > m ? m_c : m;
  double2* es = work + int64_t(e) * (5 * mm + 2 * mx * m);  // e_s
  double2* ep = es + mm;                     // e
  double2* al = ep + mm;                     // a
  double2* be = al + mm;                     // b
  double2* g = be + mm;                      // (z - e)^{-1}, then products
  double2* ag = g + mm;                      // a g
  double2* bg = ag + mx * m;                 // b g
  int* piv = reinterpret_cast<int*>(smem);
  double2* colk = reinterpret_cast<double2*>(smem + ((size_t(m) * sizeof(int) + 15) & ~size_t(15)));
  const double E = energies[e];
  const double lim = tol * scale;
  for (int i = threadIdx.x; i < mm; i += blockDim.x) {
    const int r = i / m, c = i % m;
    es[i] = ep[i] = make_double2(H00[i], 0.0);
    al[i] = make_double2(H01[i], 0.0);
    be[i] = make_double2(H01[c * m + r], 0.0);
  }
  __syncthreads();
  int it = 0;
  for (; it < max_iter; ++it) {
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      const int r = i / m, c = i % m;
      g[i] = make_double2((r == c ? E : 0.0) - ep[i].x, (r == c ? eta : 0.0) - ep[i].y);
    }
    __syncthreads();
    gj_invert<double>(g, m, m, piv, colk, status + 1);
    __syncthreads();
    cta_matmul(ag, al, g, m, m, m, false);
    cta_matmul(bg, be, g, m, m, m, false);
    cta_matmul(g, ag, be, m, m, m, false);  // a g b
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      es[i] = make_double2(es[i].x + g[i].x, es[i].y + g[i].y);
      ep[i] = make_double2(ep[i].x + g[i].x, ep[i].y + g[i].y);
    }
    __syncthreads();
    cta_matmul(g, bg, al, m, m, m, false);  // b g a
    for (int i = threadIdx.x; i < mm; i += blockDim.x) ep[i] = make_double2(ep[i].x + g[i].x, ep[i].y + g[i].y);
    __syncthreads();
    cta_matmul(g, ag, al, m, m, m, false);  // a g a
    for (int i = threadIdx.x; i < mm; i += blockDim.x) al[i] = g[i];
    __syncthreads();
    cta_matmul(g, bg, be, m, m, m, false);  // b g b
    if (threadIdx.x == 0) s_big = 0;
    __syncthreads();
    bool big = false;
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      be[i] = g[i];
      big = big || fabs(g[i].x) >= lim || fabs(g[i].y) >= lim || fabs(al[i].x) >= lim || fabs(al[i].y) >= lim;
    }
    if (big) s_big = 1;
    __syncthreads();
    const bool done = (s_big == 0);
    __syncthreads();
    if (done) break;
  }
  if (it == max_iter && threadIdx.x == 0) atomicAdd(status, 1);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) {
    const int r = i / m, c = i % m;
    g[i] = make_double2((r == c ? E : 0.0) - es[i].x, (r == c ? eta : 0.0) - es[i].y);
  }
  __syncthreads();
  gj_invert<double>(g, m, m, piv, colk, status + 1);
  __syncthreads();
  // tau (m_c x m, real) into ag as complex, then Sigma = (tau g_s) tau^T
  for (int i = threadIdx.x; i < m_c * m; i += blockDim.x) ag[i] = make_double2(tau[i], 0.0);
  __syncthreads();
  cta_matmul(bg, ag, g, m_c, m, m, false);  // tau g_s, m_c x m
  double2* o = out + int64_t(e) * stride + offset;
  for (int idx = threadIdx.x; idx < m_c * m_c; idx += blockDim.x) {
    const int i = idx / m_c, j = idx % m_c;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < m; ++k) {
      const double t = tau[j * m + k];
      re = fma(bg[i * m + k].x, t, re);
      im = fma(bg[i * m + k].y, t, im);
    }
    o[idx] = make_double2(re, im);
  }
}

size_t lead_decimation_work_elems(int m, int m_c) {
  return size_t(5) * m * m + size_t(2) * (m_c > m ? m_c : m) * m;
}

void launch_lead_decimation(const double* H00, const double* H01, const double* tau, int m, int m_c,
                            const double* energies, int n_e, double eta, double scale, double tol, int max_iter,
                            double* out, int64_t stride, int64_t offset, double* work, int* status, cudaStream_t s) {
  const size_t shm = ((size_t(m) * sizeof(int) + 15) & ~size_t(15)) + size_t(m) * sizeof(double2);
  k_lead_decimation<<<n_e, 256, shm, s>>>(H00, H01, tau, m, m_c, energies, eta, scale, tol, max_iter, (double2*)out,
                                          stride, offset, (double2*)work, status);
}

// Sigma^< = i f Gamma, Sigma^> = -i (1 - f) Gamma, Gamma = i (Sigma - Sigma^dagger)
__global__ void k_sigma_lesser(const double2* __restrict__ sr, ContactTable ct, double kT,
                               const double* __restrict__ energies, int64_t stride, double2* lesser, double2* greater) {
  const int c = blockIdx.y, e = blockIdx.z;
  const int m = ct.m[c];
  const double f = fermi_dev(energies[e], ct.mu[c], kT);
  const double2* S = sr + int64_t(e) * stride + ct.off[c];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int j = idx / m, k = idx % m;
    const double2 a = S[idx], b = S[int64_t(k) * m + j];
    const double2 dlt = make_double2(a.x - b.x, a.y + b.y);  // Sigma - Sigma^dagger = -i Gamma
    const int64_t o = int64_t(e) * stride + ct.off[c] + idx;
    if (lesser) lesser[o] = make_double2(-f * dlt.x, -f * dlt.y);
    if (greater) greater[o] = make_double2((1.0 - f) * dlt.x, (1.0 - f) * dlt.y);
  }
}

void launch_sigma_lesser(const double* sigma_r, int n_e, const ContactTable& ct, double kT, const double* energies,
                         int64_t stride, double* lesser, double* greater, cudaStream_t s) {
  k_sigma_lesser<<<dim3(16, ct.n, n_e), 256, 0, s>>>((const double2*)sigma_r, ct, kT, energies, stride,
                                                    (double2*)lesser, (double2*)greater);
}

__global__ void k_phonon(int n, int n_e, double gamma, double mu, double kT, const double* __restrict__ energies,
                         double2* r, double2* l, double2* g) {
  const int64_t tot = int64_t(n) * n_e;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < tot; i += int64_t(gridDim.x) * blockDim.x) {
    const double f = fermi_dev(energies[i / n], mu, kT);
    if (r) r[i] = make_double2(0.0, -0.5 * gamma);
    if (l) l[i] = make_double2(0.0, f * gamma);
    if (g) g[i] = make_double2(0.0, -(1.0 - f) * gamma);
  }
}

void launch_phonon(int n, int n_e, double gamma, double mu, double kT, const double* energies, double* r, double* l,
                   double* g, cudaStream_t s) {
  const int64_t tot = int64_t(n) * n_e;
  int blocks = int((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_phonon<<<blocks, 256, 0, s>>>(n, n_e, gamma, mu, kT, energies, (double2*)r, (double2*)l, (double2*)g);
}

// Self-consistent Born update of an elastic local phonon self-energy:
// Sigma_jj <- Sigma_jj + mix (D G_jj - Sigma_jj) for r, <, >.  stats[0] and
// stats[1] receive the largest |D G_jj - Sigma_jj| and the largest |D G_jj|
// through atomic maxima on their bit patterns (non-negative doubles order like
// their bits as unsigned integers).
__global__ void k_phonon_scba(int64_t tot, double D, double mix, const double2* __restrict__ Gr,
                              const double2* __restrict__ Gl, const double2* __restrict__ Gg, double2* r, double2* l,
                              double2* g, unsigned long long* stats) {
  double dmax = 0.0, smax = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < tot; i += int64_t(gridDim.x) * blockDim.x) {
    const double2* src[3] = {Gr, Gl, Gg};
    double2* dst[3] = {r, l, g};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 v = src[q][i];
      // G^< and G^> are skew-Hermitian (paper Sec. 3.1), so their diagonals are
      // purely imaginary: the rounding residue of Re is not carried into Sigma
      const double2 nw = make_double2(q == 0 ? D * v.x : 0.0, D * v.y);
      const double2 od = dst[q][i];
      const double dx = nw.x - od.x, dy = nw.y - od.y;
      dmax = fmax(dmax, hypot(dx, dy));
      smax = fmax(smax, hypot(nw.x, nw.y));
      dst[q][i] = make_double2(od.x + mix * dx, od.y + mix * dy);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(stats, (unsigned long long)__double_as_longlong(dmax));
    atomicMax(stats + 1, (unsigned long long)__double_as_longlong(smax));
  }
}

void launch_phonon_scba(int n, int n_e, double D, double mix, const double* Gr, const double* Gl, const double* Gg,
                        double* r, double* l, double* g, double* stats, cudaStream_t s) {
  const int64_t tot = int64_t(n) * n_e;
  int blocks = int((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_phonon_scba<<<blocks, 256, 0, s>>>(tot, D, mix, (const double2*)Gr, (const double2*)Gl, (const double2*)Gg,
                                       (double2*)r, (double2*)l, (double2*)g, (unsigned long long*)stats);
}

}  // namespace ndgf
