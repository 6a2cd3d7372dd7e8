// Batched FP32-pair complex GEMM on the tensor cores: C = alpha op(A) op(B) + beta D
// for the descriptors and tiles of one schedule step, like k_gemm, with the
// same results up to rounding at the FP32-pair level.
//
// Exact products of integer digits (the splitting scheme of Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59 (2012), in its fixed-point form):
//  * every row i of op(A) gets a scale 2^eA[i] >= max_k |Re a_ik| + |Im a_ik|,
//    every column j of op(B) a scale 2^eB[j] likewise (first pass of the CTA);
//  * a real x of row i becomes the integer X = round(x 2^(54 - eA[i])),
//    |X| < 2^54, written with 7 balanced base-256 digits,
//    X = sum_t d_t 256^(6-t), d_t in [-128, 127]; digits are exact in BF16;
//  * a digit product is exact (|d d'| <= 2^14) and so is the FP32 sum of up
//    to 2^10 of them, so the products of digit pair (t, t') are summed on the
//    tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate) into one
//    accumulator per group g = t + t' < 7 (pairs with t + t' >= 7 fall below
//    the 2^-54 relative resolution and are dropped), and every 8 k-steps
//    (128 terms, at most 7 * 128 * 2^14 < 2^24 per group) the groups are
//    scaled by 2^(8 (12 - g) + eA + eB - 108) and added into FP32-pair
//    accumulators;
//  * complex products use three real products, Re a Re b, Im a Im b and
//    (Re a + Im a)(Re b + Im b) (the sum formed exactly on the integers), so
//    Re = P1 - P2, Im = P3 - P1 - P2.
// The error is normwise, about 2^-54 max|a_i.| max|b_.j| k per entry: 48-bit
// accuracy for entries down to 2^-6 of their row (column) maximum, like the
// FP32-pair product on the FP32 pipe for the rest.  One CTA (8 warps) per
// 32 x 32 tile; each warp owns one m16n8 accumulator tile per group and
// component.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nd_arith.cuh"
#include "nd_internal.h"
#include "nd_kernels.h"

namespace ndgf {
namespace {

constexpr int TC_BM = 32, TC_BN = 32, TC_BK = 16;
constexpr int TC_S = 7;       // digits per real
constexpr int TC_F = 54;      // fixed-point bits below the row (column) scale
constexpr int TC_PAD = 24;    // k stride of a digit row (bf16), keeps fragment loads free of bank conflicts
constexpr int TC_FLUSH = 8;   // k-steps between two flushes of the exact FP32 group sums
constexpr int TC_NT = 256;    // threads per CTA

// shared-memory layout (bytes)
constexpr size_t TC_DIG_A = size_t(TC_S) * 3 * TC_BM * TC_PAD * 2;
constexpr size_t TC_DIG_B = size_t(TC_S) * 3 * TC_BN * TC_PAD * 2;
constexpr size_t TC_ACC = size_t(TC_NT) * 4 * 3 * sizeof(float2);  // per thread: 4 outputs x 3 products
constexpr size_t TC_SMEM = TC_DIG_A + TC_DIG_B + TC_ACC + size_t(TC_BM + TC_BN) * sizeof(int);

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower address)
  return *reinterpret_cast<const unsigned*>(&p);
}

// Balanced base-256 digits of an integer-valued float V (|V| < 2^54 after
// rounding): d[6] least significant.  Each step is exact: q = rint(V / 256)
// and V - 256 q are integers below 2^24 or multiples of the ulp of V.
__device__ __forceinline__ void digits_f(float V, float d[TC_S]) {
  V = rintf(V);
#pragma unroll
  for (int t = TC_S - 1; t > 0; --t) {
    const float q = rintf(V * 0.00390625f);
    d[t] = fmaf(q, -256.f, V);
    V = q;
  }
  d[0] = V;
}

// Brings digits in [-2^9, 2^9] back to [-128, 128] by carries toward the top.
__device__ __forceinline__ void carry(float d[TC_S]) {
#pragma unroll
  for (int t = TC_S - 1; t > 0; --t) {
    const float c = rintf(d[t] * 0.00390625f);
    d[t] = fmaf(c, -256.f, d[t]);
    d[t - 1] += c;
  }
}

// Re, Im and Re + Im of two FP32-pair complexes at consecutive k of one row
// (column) as 7 digits each (scale factor sc = 2^(54 - e)), stored as packed
// BF16 pairs at dst[(t * 3 + c) * stride] (t = 0 the most significant digit,
// c = Re, Im, Re + Im).  hi and lo parts are split separately and their
// digit sums carried; all values are integers below 2^24 in magnitude.
__device__ __forceinline__ void split_pair_store(float4 v0, float4 v1, float sc, unsigned* dst, size_t stride) {
  float r[2][TC_S], im[2][TC_S];
  const float4 v[2] = {v0, v1};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    float a[TC_S], b[TC_S];
    digits_f(v[p].x * sc, a);
    digits_f(v[p].y * sc, b);
#pragma unroll
    for (int t = 0; t < TC_S; ++t) r[p][t] = a[t] + b[t];
    carry(r[p]);
    digits_f(v[p].z * sc, a);
    digits_f(v[p].w * sc, b);
#pragma unroll
    for (int t = 0; t < TC_S; ++t) im[p][t] = a[t] + b[t];
    carry(im[p]);
  }
  float s[2][TC_S];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
#pragma unroll
    for (int t = 0; t < TC_S; ++t) s[p][t] = r[p][t] + im[p][t];
    carry(s[p]);
  }
#pragma unroll
  for (int t = 0; t < TC_S; ++t) {
    dst[(size_t(t) * 3 + 0) * stride] = pack_bf16(r[0][t], r[1][t]);
    dst[(size_t(t) * 3 + 1) * stride] = pack_bf16(im[0][t], im[1][t]);
    dst[(size_t(t) * 3 + 2) * stride] = pack_bf16(s[0][t], s[1][t]);
  }
}

__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return -70;
  int e = ilogbf(m) + 1;  // 2^e > m
  return e < -70 ? -70 : (e > 120 ? 120 : e);
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(TC_NT, 2) k_gemm_tc(const GemmDesc* __restrict__ descs, const TileRef* __restrict__ tiles,
                                                   float4* arena, int64_t se, const float4* __restrict__ aux,
                                                   int64_t sa) {
  extern __shared__ __align__(16) unsigned char sm[];
  __nv_bfloat16* Ad = reinterpret_cast<__nv_bfloat16*>(sm);             // [S][3][BM][PAD]
  __nv_bfloat16* Bd = reinterpret_cast<__nv_bfloat16*>(sm + TC_DIG_A);  // [S][3][BN][PAD]
  float2* acc_dd = reinterpret_cast<float2*>(sm + TC_DIG_A + TC_DIG_B);  // [NT][4][3]
  int* eA = reinterpret_cast<int*>(sm + TC_DIG_A + TC_DIG_B + TC_ACC);
  int* eB = eA + TC_BM;

  const TileRef tr = tiles[blockIdx.x];
  const GemmDesc d = descs[tr.desc];
  const int64_t e = blockIdx.y;
  float4* base = arena + e * se;
  const float4* abase = aux + e * sa;
  const float4* A = (d.offA & AUX_BIT) ? abase + (d.offA & ~AUX_BIT) : base + d.offA;
  const float4* B = (d.offB & AUX_BIT) ? abase + (d.offB & ~AUX_BIT) : base + d.offB;
  const int m0 = tr.tm * TC_BM, n0 = tr.tn * TC_BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool transA = d.opA != OP_N;
  const bool transB = (d.opB == OP_T || d.opB == OP_H);
  const bool conjB = (d.opB == OP_C || d.opB == OP_H);
  auto a_at = [&](int i, int k) -> float4 {  // op(A)[m0 + i][k], zero outside
    const int gm = m0 + i;
    if (gm >= d.m || k >= d.k) return make_float4(0.f, 0.f, 0.f, 0.f);
    return transA ? A[int64_t(k) * d.lda + gm] : A[int64_t(gm) * d.lda + k];
  };
  auto b_at = [&](int k, int j) -> float4 {  // op(B)[k][n0 + j], zero outside
    const int gn = n0 + j;
    if (gn >= d.n || k >= d.k) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = transB ? B[int64_t(gn) * d.ldb + k] : B[int64_t(k) * d.ldb + gn];
    if (conjB) {
      v.z = -v.z;
      v.w = -v.w;
    }
    return v;
  };

  // ---- pass 1: row and column scales over the whole k range
  if (tid < TC_BM + TC_BN) eA[tid] = 0;  // float bits of the running maxima (non-negative)
  __syncthreads();
  {  // 8 threads per row (column), each over every 8th k
    const int q = tid >> 3, part = tid & 7;
    float ma = 0.f, mb = 0.f;
    for (int k = part; k < d.k; k += 8) {
      const float4 va = a_at(q, k), vb = b_at(k, q);
      ma = fmaxf(ma, fabsf(va.x) + fabsf(va.z));
      mb = fmaxf(mb, fabsf(vb.x) + fabsf(vb.z));
    }
    atomicMax(&eA[q], __float_as_int(ma));
    atomicMax(&eB[q], __float_as_int(mb));
  }
  __syncthreads();
  if (tid < TC_BM + TC_BN) {
    // a little headroom above the hi parts: Re + Im and the lo parts stay below 2^e
    eA[tid] = scale_exp(__int_as_float(eA[tid]) * 1.0001f);
  }
  for (int64_t i = tid; i < int64_t(TC_NT) * 4 * 3; i += TC_NT) acc_dd[i] = make_float2(0.f, 0.f);
  __syncthreads();

  // ---- pass 2: digit products on the tensor cores
  const int g = lane >> 2, c4 = lane & 3;
  const int wr = (warp >> 2) * 16, wc = (warp & 3) * 8;  // warp block: rows wr.., cols wc..
  float acc[TC_S][3][4];
#pragma unroll
  for (int q = 0; q < TC_S; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[q][c][r] = 0.f;

  const int nk = (d.k + TC_BK - 1) / TC_BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int k0 = kt * TC_BK;
    // digits of the A tile (32 x 16) and the B tile (16 x 32): each thread
    // splits two consecutive k of one row of op(A) and of one column of op(B)
    {
      const int i = tid >> 3, kk = (tid & 7) * 2;
      split_pair_store(a_at(i, k0 + kk), a_at(i, k0 + kk + 1), ldexpf(1.f, TC_F - eA[i]),
                       reinterpret_cast<unsigned*>(Ad + size_t(i) * TC_PAD + kk), size_t(TC_BM) * TC_PAD / 2);
      split_pair_store(b_at(k0 + kk, i), b_at(k0 + kk + 1, i), ldexpf(1.f, TC_F - eB[i]),
                       reinterpret_cast<unsigned*>(Bd + size_t(i) * TC_PAD + kk), size_t(TC_BN) * TC_PAD / 2);
    }
    __syncthreads();
#pragma unroll
    for (int t1 = 0; t1 < TC_S; ++t1) {
      unsigned af[3][4];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const __nv_bfloat16* a0 = Ad + ((size_t(t1) * 3 + c) * TC_BM + wr + g) * TC_PAD + 2 * c4;
        af[c][0] = *reinterpret_cast<const unsigned*>(a0);
        af[c][1] = *reinterpret_cast<const unsigned*>(a0 + 8 * TC_PAD);
        af[c][2] = *reinterpret_cast<const unsigned*>(a0 + 8);
        af[c][3] = *reinterpret_cast<const unsigned*>(a0 + 8 * TC_PAD + 8);
      }
#pragma unroll
      for (int t2 = 0; t2 < TC_S - t1; ++t2) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const __nv_bfloat16* b0 = Bd + ((size_t(t2) * 3 + c) * TC_BN + wc + g) * TC_PAD + 2 * c4;
          const unsigned bf[2] = {*reinterpret_cast<const unsigned*>(b0), *reinterpret_cast<const unsigned*>(b0 + 8)};
          mma_bf16(acc[t1 + t2][c], af[c], bf);
        }
      }
    }
    __syncthreads();
    if ((kt + 1) % TC_FLUSH == 0 || kt == nk - 1) {
      // groups -> FP32-pair accumulators (each thread owns its 4 outputs)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = wr + g + (r >> 1) * 8, j = wc + 2 * c4 + (r & 1);
        const int ex = eA[i] + eB[j] - 2 * TC_F;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2& s = acc_dd[(size_t(tid) * 4 + r) * 3 + c];
          float h = s.x, lo = s.y;
#pragma unroll
          for (int q = 0; q < TC_S; ++q) {
            const float v = ldexpf(acc[q][c][r], ex + 8 * (2 * (TC_S - 1) - q));
            float sh, se2;
            two_sum(h, v, sh, se2);
            h = sh;
            lo += se2;
            acc[q][c][r] = 0.f;
          }
          s = make_float2(h, lo);
        }
      }
    }
  }
  // ---- epilogue: Re = P1 - P2, Im = P3 - P1 - P2, alpha, beta D
  float4* C = base + d.offC;
  const float4* D = base + d.offD;
  using O = Ops<DF>;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
      const int i = wr + g + (r >> 1) * 8, j = wc + 2 * c4 + (r & 1);
      const int gm = m0 + i, gn = n0 + j;
      if (gm >= d.m || gn >= d.n) continue;
      const float2* s = acc_dd + (size_t(tid) * 4 + r) * 3;
      f2 p[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) two_sum(s[c].x, s[c].y, p[c].h, p[c].l);
      float4 v = O::mk(dd_sub(p[0], p[1]), dd_sub(dd_sub(p[2], p[0]), p[1]));
      if (d.alpha == -1.0)
        v = O::neg(v);
      else if (d.alpha != 1.0)
        v = O::scale(v, d.alpha);
      if (d.beta != 0.0) {
        const float4 dv = D[int64_t(gm) * d.ldd + gn];
        v = O::add(v, d.beta == 1.0 ? dv : O::scale(dv, d.beta));
      }
      C[int64_t(gm) * d.ldc + gn] = v;
    }
}

}  // namespace

int gemm_tc_tile() { return TC_BM; }

void launch_gemm_tc(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, cudaStream_t s) {
  if (n_tiles <= 0 || w.n_e <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC_SMEM));
    attr = true;
  }
  k_gemm_tc<<<dim3(n_tiles, w.n_e), TC_NT, TC_SMEM, s>>>(d, tiles, (float4*)w.arena, w.se, (const float4*)w.aux,
                                                         w.sa);
}

}  // namespace ndgf
