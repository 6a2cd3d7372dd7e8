// Batched FP32-pair complex GEMM on the fifth-generation tensor cores
// (tcgen05): C = alpha op(A) op(B) + beta D for the descriptors of one
// schedule step, with the results of k_gemm up to rounding at the FP32-pair
// level.
//
// Products of integer digits (the splitting scheme of Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59 (2012), in its fixed-point form):
//  * every row i of op(A) gets a scale 2^eA[i] >= max_k |Re a_ik| + |Im a_ik|,
//    every column j of op(B) a scale 2^eB[j] likewise;
//  * a real x = h + l (an FP32 pair) of row i becomes the 64-bit integer
//    X = round(h 2^(54 - eA[i])) + round(l 2^(54 - eA[i])), |X| < 2^54,
//    written with 7 balanced base-256 digits (the bytes of X plus a constant
//    of 128 in every byte), X = sum_t d_t 256^(6-t), d_t in [-128, 127] and
//    |d_0| <= 64; digit t is
//    held as d_t 2^(-8t), exact in BF16 (8 significant bits, a power-of-two
//    weight), so a product of digits t, t' carries its weight 2^(-8(t+t'));
//  * the 28 pairs with t + t' <= 6 are kept (the rest lie below the 2^-54
//    resolution); the products of each group g = t + t' = 0 .. 3 are summed
//    in an FP32 accumulator of their own in TMEM, exactly (a group sum is an
//    integer times its weight, at most 3 2^14 per k, so below 2^24 over CHUNK
//    16-k blocks), and groups 4, 5, 6, whose weights are 2^-32 .. 2^-48 of
//    the top, share a fifth accumulator whose FP32 rounding stays near 2^-53
//    of the result (sharing from group 3 on would cost 2^-44);
//  * complex products take three real products, Re a Re b, Im a Im b and
//    (Re a + Im a)(Re b + Im b) (the sum formed exactly on the 64-bit integers), so
//    Re = P1 - P2, Im = P3 - P1 - P2.
// The error is normwise, about 2^-52 max|a_i.| max|b_.j| k per entry.
//
// Two kernels per launch:
//  * k_tc_split: the scale and the digits of Re, Im and Re + Im of every row
//    of op(A) and column of op(B) of every descriptor, once, into a per-energy
//    scratch as weighted BF16 digit planes in the tensor cores' K-major
//    core-matrix layout (core matrices of 8 rows x 8 k, no swizzle), so that
//    the 7 planes of one tile and 16 k are one contiguous block;
//  * k_gemm_tc: one CTA per 128 x 64 output tile and energy, warp-specialised.
//    A producer warp streams the planes of each job (16 k of one component)
//    into a 4-stage shared-memory ring with bulk asynchronous copies
//    (cp.async.bulk, completion by mbarrier transaction count).  One thread
//    issues the 28 digit-pair MMAs per job (tcgen05.mma kind::f16, M = 128,
//    N = 64, K = 16, both operands from shared memory, FP32 accumulators in
//    TMEM) into NACC 64-column accumulators; tcgen05.commit frees the stages.
//    At the end of every chunk (CHUNK 16-k blocks, or a component) sixteen
//    accumulator warps read the accumulators (tcgen05.ld), add them into
//    FP32-pair accumulators of Re and Im in registers (16 outputs per
//    thread) and hand them back.  The epilogue stages the tile in shared
//    memory and writes rows of C with coalesced stores, the loads of D for
//    8 rows per warp in flight together.
// Every wait is bounded.  A wait that gives up raises the CTA's abort flag;
// the CTA then drains its copies and MMAs, frees its TMEM, skips its output
// and sets *timeout (reported by nd_fact_status as ND_ERR_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nd_arith.cuh"
#include "nd_internal.h"
#include "nd_kernels.h"

namespace ndgf {
namespace {

constexpr int TC_S = TC_DIGITS;  // digits per real
constexpr int TC_F = 54;         // fixed-point bits below the row (column) scale
static_assert(TC_S == 7, "the byte layout of the digits assumes 7 digits per real");
constexpr int NACC = 5;          // TMEM accumulators: groups 0, 1, 2, 3 and 4..6
constexpr int ACC_COLS = NACC * TC_N;
// One stage (a job: 16 k of one component): the 7 weighted BF16 digit planes
// of the tile's rows of op(A) and of its columns of op(B), in the tensor
// cores' K-major core-matrix layout, as the split wrote them.
constexpr int PA = 2 * int(TC_PLANE_A), PB = 2 * int(TC_PLANE_B);  // bytes of one BF16 plane
constexpr int SA = TC_S * PA, SB = TC_S * PB;
constexpr int STAGES = 4;        // shared-memory stages (bulk copies)
constexpr int TMEM_COLS = 512;   // allocated (a power of two): the accumulators
constexpr int CHUNK = 20;     // 16-k blocks summed in TMEM between two reads (320 terms: group sums < 2^24)
constexpr int FW = 16;        // accumulator warps: flush and epilogue
constexpr int CPT = TC_N / (FW / 4);  // accumulator columns per thread (4 warps per TMEM lane quadrant)
constexpr int NT = (FW + 2) * 32;     // + producer warp + MMA warp
constexpr size_t SMEM = size_t(STAGES) * (SA + SB) + 1024;  // + alignment slack
constexpr long SPIN = 1L << 25;    // polls before a wait gives up (default; a drain always uses it)
constexpr int TILE_LD = TC_N + 1;  // float4 row stride of the output tile staged in shared memory
constexpr int EPI_ROWS = TC_M / FW;  // output rows per warp, their D loads in flight together

static_assert(ACC_COLS <= TMEM_COLS, "accumulators exceed the TMEM columns");
static_assert(size_t(TC_M) * TILE_LD * 16 <= size_t(STAGES) * (SA + SB), "the output tile must fit in the stages");
static_assert(CPT % 4 == 0 && TC_M % FW == 0, "accumulator warp layout");
static_assert(CHUNK * 16 * 3 * (1 << 14) < (1 << 24), "group sums of a chunk must stay exact in FP32");
static_assert(TC_M == 128 && TC_N % 16 == 0 && TC_N <= 256, "tcgen05 kind::f16 shape with M = 128");

// Four signed bytes of w (byte 0 first) times the power of two wt as two
// packed BF16 pairs, without conversion instructions: with u = w ^ 0x80808080
// every byte is b = d + 128 in [0, 255]; the float with bits 0x4B0000bb is
// 2^23 + b exactly, so fma(x, wt, -(2^23 + 128) wt) = d wt exactly, a value
// with at most 8 significant bits, whose upper 16 bits are its BF16 form.
__device__ __forceinline__ uint2 widen4(unsigned w, float wt, float off) {
  const unsigned u = w ^ 0x80808080u;
  const float f0 = fmaf(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7650)), wt, off);
  const float f1 = fmaf(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7651)), wt, off);
  const float f2 = fmaf(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7652)), wt, off);
  const float f3 = fmaf(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7653)), wt, off);
  return make_uint2(__byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632),
                    __byte_perm(__float_as_uint(f2), __float_as_uint(f3), 0x7632));
}

// The fixed-point integer of one FP32 pair (h, l) of a row with scale factor
// sc = 2^(54 - e): X = round(h sc) + round(l sc), |X| < 2^54 (the products by
// the power of two sc are exact, the conversions round to nearest).
__device__ __forceinline__ long long fixed_of(float h, float l, float sc) {
  return __float2ll_rn(h * sc) + __float2ll_rn(l * sc);
}

// Balanced base-256 digits of X, |X| < 2^54, as two's-complement bytes:
// Y = X + sum_{b < 7} 128 256^b lies in [0, 2^56), so X = sum_b (y_b - 128) 256^b
// with the bytes y_b of Y; digit t = y_(6-t) - 128 is in [-128, 127] (and in
// [-64, 64] for t = 0), and its byte is y_(6-t) xor 0x80.  Byte b of the
// result (b < 7) holds digit 6 - b; lo = bytes 0..3, hi = bytes 4..6.
__device__ __forceinline__ void digit_bytes(long long X, unsigned& lo, unsigned& hi) {
  const unsigned long long y = (unsigned long long)(X + 0x80808080808080LL) ^ 0x80808080808080ULL;
  lo = unsigned(y);
  hi = unsigned(y >> 32);
}

// 4 x 4 byte transpose: out[b] byte q = in[q] byte b.
__device__ __forceinline__ void transpose4(const unsigned (&in)[4], unsigned (&out)[4]) {
  const unsigned t0 = __byte_perm(in[0], in[1], 0x5140), t1 = __byte_perm(in[0], in[1], 0x7362);
  const unsigned t2 = __byte_perm(in[2], in[3], 0x5140), t3 = __byte_perm(in[2], in[3], 0x7362);
  out[0] = __byte_perm(t0, t2, 0x5410);
  out[1] = __byte_perm(t0, t2, 0x7632);
  out[2] = __byte_perm(t1, t3, 0x5410);
  out[3] = __byte_perm(t1, t3, 0x7632);
}

// The fixed-point integer of component c of an FP32-pair complex (c = 0: Re,
// 1: Im, 2: Re + Im, the integer sum X_re + X_im, |X| < 2^54 as the row scale
// bounds |Re| + |Im|).
__device__ __forceinline__ long long comp_fixed(const float4& v, float sc, int c) {
  const long long xr = c != 1 ? fixed_of(v.x, v.y, sc) : 0;
  const long long xi = c != 0 ? fixed_of(v.z, v.w, sc) : 0;
  return xr + xi;
}

// Digits of component c of 8 FP32-pair complexes at consecutive k of one row
// (scale factor sc) into w[t][0..1]: the 8 bytes of digit plane t, element q
// at byte q.
__device__ __forceinline__ void split8(const float4 (&v)[8], float sc, int c, unsigned (&w)[TC_S][2]) {
  unsigned lo[8], hi[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) digit_bytes(comp_fixed(v[q], sc, c), lo[q], hi[q]);
#pragma unroll
  for (int g = 0; g < 2; ++g) {  // elements 4g .. 4g + 3: word g of every plane
    const unsigned il[4] = {lo[4 * g], lo[4 * g + 1], lo[4 * g + 2], lo[4 * g + 3]};
    const unsigned ih[4] = {hi[4 * g], hi[4 * g + 1], hi[4 * g + 2], hi[4 * g + 3]};
    unsigned ol[4], oh[4];
    transpose4(il, ol);
    transpose4(ih, oh);
#pragma unroll
    for (int b = 0; b < 4; ++b) w[TC_S - 1 - b][g] = ol[b];
#pragma unroll
    for (int b = 0; b < 3; ++b) w[TC_S - 5 - b][g] = oh[b];
  }
}

__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return -70;
  int e = ilogbf(m) + 1;  // 2^e > m
  return e < -70 ? -70 : (e > 120 ? 120 : e);
}

// Byte offset of element (r, k), k < 16, in a BF16 digit plane in the
// tensor cores' K-major layout without swizzle: core matrices of 8 rows x 8 k
// take 16 bytes per row and 128 bytes each, the two core matrices of a row
// group along k are 128 bytes apart (leading byte offset) and consecutive row
// groups 256 bytes (stride byte offset).
__host__ __device__ constexpr uint32_t core_off(int r, int k) {
  return uint32_t((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t CORE_LBO = 128, CORE_SBO = 256;

// ---- split: one CTA per 32 rows of op(A) or columns of op(B); lane = row,
// warp w takes the k octets w, w + 8, ...
__global__ void __launch_bounds__(256, 4) k_tc_split(const GemmDesc* __restrict__ descs, const TcDesc* __restrict__ tcd,
                                                  const TcSplit* __restrict__ items, const float4* __restrict__ arena,
                                                  int64_t se, const float4* __restrict__ aux, int64_t sa,
                                                  unsigned char* __restrict__ scratch, int64_t ss) {
  __shared__ float red[8][32];
  const TcSplit it = items[blockIdx.x];
  const TcDesc t = tcd[it.tcd];
  const GemmDesc d = descs[t.desc];
  const int64_t e = blockIdx.y;
  const bool side_a = it.side == 0;
  const int64_t off = side_a ? d.offA : d.offB;
  const float4* X = (off & AUX_BIT) ? aux + e * sa + (off & ~AUX_BIT) : arena + e * se + off;
  const int64_t ld = side_a ? d.lda : d.ldb;
  // element (r, k) of op(A), or of op(B)^T, sits at X[r ld + k] (row major) or X[k ld + r]
  const bool row_major = side_a ? d.opA == OP_N : (d.opB == OP_T || d.opB == OP_H);
  const bool cj = !side_a && (d.opB == OP_C || d.opB == OP_H);
  const int rows = side_a ? d.m : d.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = it.r0 + lane;
  const bool live = r < rows;
  auto at = [&](int k) -> float4 {
    if (!live || k >= d.k) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = row_major ? X[int64_t(r) * ld + k] : X[int64_t(k) * ld + r];
    if (cj) {
      v.z = -v.z;
      v.w = -v.w;
    }
    return v;
  };
  const int n_oct = 2 * t.kb;
  float mx = 0.f;
  for (int o = w; o < n_oct; o += 16) {  // two octets per pass: 16 loads in flight
    float4 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = at(8 * o + (q < 8 ? q : 56 + q));
#pragma unroll
    for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fabsf(v[q].x) + fabsf(v[q].z));
  }
  red[w][lane] = mx;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) mx = fmaxf(mx, red[i][lane]);
  // a little headroom above the hi parts: Re + Im and the lo parts stay below 2^e
  const int ex = scale_exp(mx * 1.0001f);
  unsigned char* scr = scratch + e * ss;
  if (w == 0) reinterpret_cast<int*>(scr)[(side_a ? t.exp_a : t.exp_b) + r] = ex;
  const float sc = ldexpf(1.f, TC_F - ex);
  const int R = side_a ? TC_M : TC_N, RB = side_a ? t.rba : t.rbb;
  const int64_t P = side_a ? PA : PB;  // bytes of a BF16 plane
  unsigned char* dig = scr + (side_a ? t.dig_a : t.dig_b);
  const int rb = r / R, rr = r - rb * R;
  for (int o = w; o < n_oct; o += 8) {
    const int kb = o >> 1, k0 = o * 8;
    float4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = at(k0 + q);
    const uint32_t co = core_off(rr, (o & 1) * 8);
#pragma unroll
    for (int c = 0; c < 3; ++c) {  // one component at a time: fewer live registers
      unsigned wd[TC_S][2];
      split8(v, sc, c, wd);
#pragma unroll
      for (int tt = 0; tt < TC_S; ++tt) {
        const float wt = __int_as_float((127 - 8 * tt) << 23);  // digit weight 2^(-8t)
        const float wo = -8388736.f * wt;                        // -(2^23 + 128) wt, exact
        const uint2 lo = widen4(wd[tt][0], wt, wo), hi = widen4(wd[tt][1], wt, wo);
        unsigned char* pl = dig + (((int64_t(c) * t.kb + kb) * RB + rb) * TC_S + tt) * P + co;
        *reinterpret_cast<uint4*>(pl) = make_uint4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  }
}

// ---- PTX wrappers (tcgen05, mbarrier, bulk copies)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity.  Gives up when the CTA's
// abort flag is raised (checked every 64 polls) or after `spin` polls (then
// raises it).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, long spin) {
  for (long i = 0; i < spin; ++i) {
    if (mbar_try(b, parity)) return true;
    if ((i & 63) == 63 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
// Bounded wait that ignores the abort flag: for work that completes by
// itself (copies and MMAs in flight) before shared memory or TMEM is released.
__device__ __forceinline__ bool mbar_drain(uint64_t* b, uint32_t parity) {
  for (long i = 0; i < SPIN; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((CORE_LBO >> 4) & 0x3FFF) << 16) |
         (uint64_t((CORE_SBO >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TC_N >> 3) << 17) |
                           (uint32_t(TC_M >> 4) << 24);

// D (TMEM) (+)= A B, both operands in shared memory (matrix descriptors)
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}
// barrier over the first `count` threads (whole warps) of the CTA
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// (H, L) += (h, l), unnormalised pairs
__device__ __forceinline__ void dd_acc(float& H, float& L, float h, float l) {
  float s, err;
  two_sum(H, h, s, err);
  H = s;
  L += err + l;
}

__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const GemmDesc* __restrict__ descs, const TcDesc* __restrict__ tcd,
                                                   const TileRef* __restrict__ tiles, float4* arena, int64_t se,
                                                   const unsigned char* __restrict__ scratch, int64_t ss,
                                                   int* timeout, long spin) {
  extern __shared__ unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accfull, accempty, done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int eA[TC_M], eB[TC_N];
  unsigned char* ring = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);  // STAGES x (SA + SB) bytes

  const TileRef tr = tiles[blockIdx.x];
  const TcDesc t = tcd[tr.desc];
  const GemmDesc d = descs[t.desc];
  const int64_t e = blockIdx.y;
  const unsigned char* scr = scratch + e * ss;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accfull, 1);
    mbar_init(&accempty, FW);
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abrt = &abort_flag;
  const int KB = t.kb, njobs = 3 * KB;  // job j: component j / KB, 16-k block j % KB

  if (warp == FW) {
    // ---- producer: the BF16 digit planes of A and B of each job into the stages
    if (lane == 0) {
      auto plane_a = [&](int jj) {
        const int c = jj / KB, kb = jj - c * KB;
        return scr + t.dig_a + ((int64_t(c) * KB + kb) * t.rba + tr.tm) * int64_t(SA);
      };
      auto plane_b = [&](int jj) {
        const int c = jj / KB, kb = jj - c * KB;
        return scr + t.dig_b + ((int64_t(c) * KB + kb) * t.rbb + tr.tn) * int64_t(SB);
      };
      int j = 0;
      for (; j < njobs; ++j) {
        const int s = j % STAGES, u = j / STAGES;
        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, abrt, spin)) break;
        unsigned char* st = ring + size_t(s) * (SA + SB);
        mbar_expect_tx(&full[s], SA + SB);
        bulk_g2s(st, plane_a(j), SA, &full[s]);
        bulk_g2s(st + SA, plane_b(j), SB, &full[s]);
      }
      // the last copies into every stage have landed before the CTA ends
      for (int jj = j > STAGES ? j - STAGES : 0; jj < j; ++jj) mbar_drain(&full[jj % STAGES], (jj / STAGES) & 1);
    }
  } else if (warp == FW + 1) {
    // ---- MMA issue: 28 digit-pair products per job into the group accumulators
    if (lane == 0) {
      int q = 0;  // chunks handed to the accumulator warps
      for (int j = 0; j < njobs; ++j) {
        const int s = j % STAGES, u = j / STAGES;
        const int kb = j % KB, kc = kb % CHUNK;
        if (kc == 0 && q > 0) {  // the accumulators were read back by the accumulator warps
          if (!mbar_wait(&accempty, (q - 1) & 1, abrt, spin)) break;
          tc_fence_after();
        }
        // the bulk copies of this stage have landed (the wait acquires their writes)
        if (!mbar_wait(&full[s], u & 1, abrt, spin)) break;
        const uint32_t sa = smem_u32(ring + size_t(s) * (SA + SB)), sb = sa + SA;
#pragma unroll
        for (int t1 = 0; t1 < TC_S; ++t1)
#pragma unroll
          for (int t2 = 0; t2 < TC_S - t1; ++t2) {
            const int acc = t1 + t2 < NACC - 1 ? t1 + t2 : NACC - 1;
            // the first product into each accumulator of a chunk overwrites it
            const uint32_t accumulate = (kc == 0 && t1 == 0 && t2 <= NACC - 1) ? 0u : 1u;
            mma_bf16(tmem + uint32_t(acc * TC_N), sdesc(sa + uint32_t(t1 * PA)), sdesc(sb + uint32_t(t2 * PB)), accumulate);
          }
        if (j + STAGES < njobs) mma_commit(&empty[s]);
        if (kc == CHUNK - 1 || kb == KB - 1) {
          mma_commit(&accfull);
          ++q;
        }
      }
      // every MMA issued has completed before the TMEM is released
      mma_commit(&done);
      mbar_drain(&done, 0);
    }
  } else {
    // ---- accumulator warps: after every chunk read the TMEM lanes 32 (warp % 4) ..,
    // columns CPT (warp / 4) .. and fold them into FP32-pair accumulators
    const int quad = warp & 3, cg = warp >> 2;
    const uint32_t tbase = tmem + (uint32_t(quad * 32) << 16) + uint32_t(cg * CPT);
    float ac[CPT][4];  // Re (hi, lo), Im (hi, lo) of CPT outputs, unnormalised pairs
#pragma unroll
    for (int o = 0; o < CPT; ++o) ac[o][0] = ac[o][1] = ac[o][2] = ac[o][3] = 0.f;
    const int nch = (KB + CHUNK - 1) / CHUNK;
    bool ok = true;
    int q = 0;  // chunks flushed
    for (int c = 0; c < 3 && ok; ++c) {
      for (int ch = 0; ch < nch; ++ch, ++q) {
        ok = __all_sync(0xffffffffu, mbar_wait(&accfull, q & 1, abrt, spin));
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int cs = 0; cs < CPT; cs += 4) {
          float v[NACC][4];
#pragma unroll
          for (int g = 0; g < NACC; ++g) tmem_ld4(tbase + uint32_t(g * TC_N + cs), v[g]);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            // P = the sum of the (already weighted) accumulators as an unnormalised pair
            float h = v[0][i], l = 0.f;
#pragma unroll
            for (int g = 1; g < NACC; ++g) {
              float sum, err;
              two_sum(h, v[g][i], sum, err);
              h = sum;
              l += err;
            }
            float* a = ac[cs + i];
            if (c == 0) {  // Re += P1, Im -= P1
              dd_acc(a[0], a[1], h, l);
              dd_acc(a[2], a[3], -h, -l);
            } else if (c == 1) {  // Re -= P2, Im -= P2
              dd_acc(a[0], a[1], -h, -l);
              dd_acc(a[2], a[3], -h, -l);
            } else {  // Im += P3
              dd_acc(a[2], a[3], h, l);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty);
      }
    }
    // ---- epilogue through shared memory, which is idle once the last chunk
    // has been read (every copy consumed, every MMA complete): each thread
    // puts its CPT outputs, scaled by 2^(eA + eB - 12) (the weighted digits
    // carry 2^96 of the 2^-108) as 2^(eA - 6) 2^(eB - 6), into a padded
    // 128 x 64 tile; then whole warps write rows of C (alpha, beta D) with
    // consecutive lanes on consecutive columns.  A warp that gave up has
    // raised the abort flag before the first barrier, so no warp writes C then.
    float4* tile = reinterpret_cast<float4*>(ring);  // [TC_M][TILE_LD]
    {  // the row and column exponents, loaded only now so that the start of the CTA does not wait for them
      const int* xa = reinterpret_cast<const int*>(scr) + t.exp_a + int64_t(tr.tm) * TC_M;
      const int* xb = reinterpret_cast<const int*>(scr) + t.exp_b + int64_t(tr.tn) * TC_N;
      for (int i = tid; i < TC_M; i += FW * 32) eA[i] = xa[i];
      for (int i = tid; i < TC_N; i += FW * 32) eB[i] = xb[i];
    }
    named_sync(1, FW * 32);
    if (ok) {
      const int row = quad * 32 + lane;
      const float fa = __int_as_float((eA[row] - 6 + 127) << 23);
#pragma unroll
      for (int o = 0; o < CPT; ++o) {
        const int jl = cg * CPT + o;
        const float f = fa * __int_as_float((eB[jl] - 6 + 127) << 23);
        f2 re, im;
        two_sum(ac[o][0], ac[o][1], re.h, re.l);
        two_sum(ac[o][2], ac[o][3], im.h, im.l);
        tile[row * TILE_LD + jl] = make_float4(re.h * f, re.l * f, im.h * f, im.l * f);
      }
    }
    named_sync(1, FW * 32);
    if (!*abrt) {
      using O = Ops<DF>;
      const int gm0 = tr.tm * TC_M, gn0 = tr.tn * TC_N;
      float4* C = arena + e * se + d.offC + int64_t(gm0) * d.ldc + gn0;
      const float4* D = arena + e * se + d.offD + int64_t(gm0) * d.ldd + gn0;
      const int rows = min(TC_M, d.m - gm0), cols = min(TC_N, d.n - gn0);
      const int amode = d.alpha == 1.0 ? 0 : (d.alpha == -1.0 ? 1 : 2);
      const int bmode = d.beta == 0.0 ? 0 : (d.beta == 1.0 ? 1 : 2);
      const int r0 = warp * EPI_ROWS;  // this warp's rows, their D loads in flight together
      float4 dv[EPI_ROWS][TC_N / 32];
      if (bmode) {
#pragma unroll
        for (int i = 0; i < EPI_ROWS; ++i)
#pragma unroll
          for (int h2 = 0; h2 < TC_N / 32; ++h2) {
            const int r = r0 + i, jl = h2 * 32 + lane;
            dv[i][h2] = (r < rows && jl < cols) ? D[int64_t(r) * d.ldd + jl] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
      }
#pragma unroll
      for (int i = 0; i < EPI_ROWS; ++i)
#pragma unroll
        for (int h2 = 0; h2 < TC_N / 32; ++h2) {
          const int r = r0 + i, jl = h2 * 32 + lane;
          if (r < rows && jl < cols) {
            float4 v = tile[r * TILE_LD + jl];
            if (amode == 1)
              v = O::neg(v);
            else if (amode == 2)
              v = O::scale(v, d.alpha);
            if (bmode) v = O::add(v, bmode == 1 ? dv[i][h2] : O::scale(dv[i][h2], d.beta));
            C[int64_t(r) * d.ldc + jl] = v;
          }
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (tid == 0 && abort_flag) atomicExch(timeout, 1);
}

}  // namespace

void prepare_gemm_tc() { cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM)); }

int64_t gemm_tc_scratch(const GemmDesc& g, TcDesc& t, int64_t off) {
  t.kb = (g.k + 15) / 16;
  t.rba = (g.m + TC_M - 1) / TC_M;
  t.rbb = (g.n + TC_N - 1) / TC_N;
  t.dig_a = off;
  off += 3 * int64_t(t.kb) * t.rba * SA;
  t.dig_b = off;
  off += 3 * int64_t(t.kb) * t.rbb * SB;
  t.exp_a = off / 4;
  off += int64_t(t.rba) * TC_M * 4;
  t.exp_b = off / 4;
  off += int64_t(t.rbb) * TC_N * 4;
  return (off + 1023) & ~int64_t(1023);
}

void launch_gemm_tc(const Work& w, const GemmDesc* d, const TcDesc* tcd, const TcSplit* splits, int n_splits,
                    const TileRef* tiles, int n_tiles, unsigned char* scratch, int64_t ss, int* timeout,
                    int64_t wait_polls, cudaStream_t s) {
  if (n_tiles <= 0 || w.n_e <= 0) return;
  if (n_splits > 0)
    k_tc_split<<<dim3(n_splits, w.n_e), 256, 0, s>>>(d, tcd, splits, (const float4*)w.arena, w.se,
                                                     (const float4*)w.aux, w.sa, scratch, ss);
  const long spin = wait_polls > 0 ? long(wait_polls) : SPIN;
  k_gemm_tc<<<dim3(n_tiles, w.n_e), NT, SMEM, s>>>(d, tcd, tiles, (float4*)w.arena, w.se, scratch, ss, timeout,
                                                   spin);
}

}  // namespace ndgf
