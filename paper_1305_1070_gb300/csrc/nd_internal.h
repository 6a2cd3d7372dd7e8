// Internal structures shared by the host planner (nd_plan.cpp) and the CUDA
// side (nd_api.cu, nd_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ndgf.h"

namespace ndgf {

// Thread-local error message for nd_last_error().
void set_error(const std::string& msg);
nd_status fail(nd_status st, const std::string& msg);

// One cluster of the nested-dissection tree (paper Sec. 3.2).  Clusters are
// stored in postorder: every descendant of a cluster precedes it.
struct Cluster {
  int level = 0;      // 1 = leaf; a cluster's level is 1 + max(level of children)
  int parent = -1;    // -1 = root
  int slot = 0;       // index of this cluster among its parent's children
  int first_desc = 0; // postorder index of the first cluster of its subtree
  int n = 0, b = 0;   // rows eliminated here, size of the boundary B_i
  // Delayed pivots (nd_opts.delay): k rows of the front are not eliminated
  // here but passed on to the parent, where they are the k "virtual" unknowns
  // starting at front row dslot.  Which k rows are delayed is decided per
  // energy (k_delay); the front then holds the eliminated rows first.  The
  // front has n + k rows: n_own own sites, then the children's virtual rows.
  int k = 0, n_own = 0, dslot = -1;
  int nf() const { return n + k; }
  std::vector<int> I; // front rows: own sites (caller ids, contact sites first), then virtual ids (>= n_sites)
  std::vector<int> B; // boundary: own virtual ids (k, in the parent), then ancestor sites coupled after folding
  std::vector<int> map; // B[k] -> position in the parent's front [I_p ; B_p]
  std::vector<std::pair<int, int>> contacts; // (contact id, first row in I)
  std::vector<int> children;
  bool nactive = false; // the subtree holds a contact (N of Sec. 3.2 nonzero without phonons)
  int A = 0;            // number of sites of all ancestors (columns of the extended blocks)
  // per-energy workspace regions, offsets in complex elements
  int64_t off_F = 0;    // (n+k) x (n+b): [A_ii | A_iB] folded front; A_ii^{-1} after the fold
  int64_t off_Psi = 0;  // n x b   : Psi_i = -A_ii^{-1} A_iB
  int64_t off_BB = 0;   // b x b   : Schur update accumulator, then G_BB
  int64_t off_G = 0;    // n x (n+b): [G_II | G_IB]; (n+k) x (n+b) scratch of k_delay during the fold
  int64_t off_PBB[2] = {0, 0}; // b x b: P_BB for Sigma^< (0) and Sigma^> (1)
  int64_t off_P[2] = {0, 0};   // n x (n+b): [P_II | P_IB]
  // G^< workspace of clusters whose row block of N is nonzero, per variant
  // (0: contacts only, 1: every cluster), -1 when the cluster has none.
  // Columns run over Y_i = I_i followed by all ancestor sites (nearest first).
  struct Ext {
    int64_t off_GX = -1;       // n x A      : G_{I_i, anc(i)}
    int64_t off_GBA = -1;      // b x A      : G_{B_i, anc(i)} (gathered)
    int64_t off_NX[2] = {-1, -1}; // n x (n+A): N_{I_i, Y_i}
    int64_t off_NB[2] = {-1, -1}; // b x A    : fold accumulator N_{B_i, anc(i)}
    int64_t off_PX[2] = {-1, -1}; // n x (n+A): A_ii^{-1} N_{I_i, Y_i}
  } ext[2];
  // adjoint solves (nd_density_gradient), offsets relative to the adjoint
  // part of the workspace, M columns = all contact sites:
  // XI (n x M) right-hand side / upward accumulator, RB (b x M) boundary
  // updates, XB (b x M) gathered boundary solution, XS (n x M) solution,
  // U (n x M) solution of the first solve
  int64_t adj_XI = 0, adj_RB = 0, adj_XB = 0, adj_XS = 0, adj_U = 0;
};

// ---- device descriptors (plain structs, copied to the GPU) -----------------
struct AssembleDesc {
  int64_t off_F, off_BB;
  int32_t n, b, ld;          // n = front rows, b = boundary, ld = row length of F
  int32_t n_own;             // rows with a site of their own (the rest are virtual)
  int32_t ent_begin, ent_end; // range in the assembly entry list
  int32_t site_begin;        // range [site_begin, site_begin+n) of the site list
  int32_t c0, m0, soff0;     // first contact: row offset, size, offset in packed Sigma (elements)
  int32_t c1, m1, soff1;     // second contact (m1 = 0 if none)
};

struct InvDesc {
  int64_t off;  // matrix start (row major, leading dimension ld)
  int32_t n, ld;
  int32_t cluster;
  int32_t fp64; // 1: invert in complex128 even on the mixed path
  int64_t scr;  // fp64 blocks: offset of this block's complex128 scratch within an energy's
};

enum : int32_t { OP_N = 0, OP_T = 1, OP_C = 2, OP_H = 3 };

// C = alpha * op(A) * op(B) + beta * D.  Offsets are per-energy element
// offsets into the workspace; a set bit 62 selects the auxiliary buffer.
struct GemmDesc {
  int64_t offA, offB, offC, offD;
  int32_t m, n, k;
  int32_t lda, ldb, ldc, ldd;
  int32_t opA, opB;
  double alpha, beta;
};
static constexpr int64_t AUX_BIT = int64_t(1) << 62;

// Extend-add of a child's b_c x b_c update into the parent's front
// (rows in I_p -> front [n_p x (n_p+b_p)], rows and columns in B_p -> BB).
struct ScatterDesc {
  int64_t off_src;   // child's b x b block
  int64_t off_front; // parent's front, rows of length n_p + b_p
  int64_t off_bb;    // parent's b_p x b_p block
  int32_t b, n_p, b_p;
  int32_t map_begin; // child's map in the map array
  int32_t k_p;       // parent's delayed rows: front rows are map positions < n_p + k_p
};

// Gather of a child's G_BB (or P_BB) from its parent's front.
struct GatherDesc {
  int64_t off_dst;   // child's b x b block
  int64_t off_front; // parent's [X_II | X_IB]
  int64_t off_bb;    // parent's X_BB
  int32_t b, n_p, b_p;
  int32_t map_begin;
  int32_t k_p, sb_p; // parent's delayed rows and first unknown (per-energy row order)
};

struct DiagDesc {
  int64_t off;      // n x ld block
  int32_t n, ld;
  int32_t site_begin;
};

struct NPhDesc {     // N_{I,Y} = diag(ph) conj([G_II | G_{I,anc}]) for one cluster and one side
  int64_t off_NX, off_G, off_GX;
  int32_t n, ldG, A;  // N is n x (n + A); G front has leading dimension ldG
  int32_t site_begin;
  int32_t rhs;        // 0: Sigma^<_ph, 1: Sigma^>_ph
};

// G_{B_i, anc(i)}: entry (r, j) is G between B_i[r] and the j-th ancestor site,
// read from the G_II block or the extended block of the lower of the two
// owning clusters (G^r is complex symmetric).
struct AncGatherDesc {
  int64_t off_dst;   // b x A
  int32_t b, A;
  int32_t bsite_begin;   // B_i unknowns in the unknown-id array
  int32_t anc_begin;     // ancestor columns (cluster, row) in the anc arrays
};

// Rows of a child's fold update C (b x A_c, columns = Y_parent) into the
// parent's N (rows in I_p) or its accumulator (rows in B_p, columns anc(p)).
struct RowScatterDesc {
  int64_t off_src, off_nx, off_nb;
  int32_t b, A_c, n_p, A_p;
  int32_t map_begin;
  int32_t k_p, sb_p; // parent's delayed rows and first unknown (per-energy row order)
};

// Delayed-pivot selection of one cluster (k_delay): front F with nf = n + k
// rows of length ld, boundary accumulator BB (bb x bb, bb = b), scratch S in
// the G region; unknowns [sb, sb + nf) of the cluster, the parent's virtual
// rows of this cluster start at unknown sb_p + dslot.
struct DelayDesc {
  int64_t off_F, off_BB, off_S;
  int32_t nf, k, ld, bb;
  int32_t sb, sb_p, dslot;
};

// Row moves of the adjoint solves between a child's b x M block and its
// parent's interior (m_p x M) and boundary (b_p x M) blocks, through the map
// of the child's boundary into the parent's front (per-energy row order of
// the parent when it has delayed rows).
struct RowsDesc {
  int64_t off_child;  // child's b x M block
  int64_t off_pi;     // parent's interior block (m_p x M)
  int64_t off_pb;     // parent's boundary block (b_p x M)
  int32_t b, m_p, k_p, sb_p;
  int32_t map_begin;
};

// Per-cluster blocks of the adjoint solves (absolute per-energy offsets).
struct AdjDesc {
  int64_t off_XI, off_RB, off_XS, off_U;
  int32_t m, b, site_begin, pad;
};

// Final position of every front row after the delayed pivots (k_loc).
struct LocDesc {
  int32_t sb, nf, n;  // first unknown, front rows, rows eliminated here
  int32_t cluster;
  int32_t sb_p, dslot; // parent's first unknown and this cluster's virtual rows there
};

// P_{I,F}[:, j] = PX[:, cmap[j]] (columns I_i then B_i picked out of Y_i).
struct ColGatherDesc {
  int64_t off_P, off_PX;
  int32_t n, b, A;
  int32_t cmap_begin;
  int32_t bsite_begin;   // B_i unknowns (used with per-energy positions)
};

struct ZeroDesc {
  int64_t off;
  int64_t count;
};

// Per-cluster geometry used by the S9 certificate to find a stored entry.
struct CertCluster {
  int64_t offG, offP, offPg; // [G_II | G_IB] and [P_II | P_IB] fronts of G^< and G^>
  int32_t sb, n, ld;         // first unknown slot, rows eliminated here, row length n + b
  int32_t parent, dslot;     // parent (-1: root) and this cluster's virtual rows in the parent's front
  int32_t first_desc;        // postorder index of the first cluster of the subtree
  int32_t bs, b;             // sorted boundary slots: cert_bslot[bs .. bs + b)
};

// A launch of the precomputed schedule.
enum StepKind : int32_t {
  ST_INVERSE = 0,
  ST_GEMM = 1,
  ST_SCATTER = 2,
  ST_GATHER_SYM = 3,
  ST_GATHER_SKEW = 4,
  ST_ZERO = 5,
  ST_NPH = 6,
  ST_GATHER_ANC = 7,
  ST_SCATTER_ROWS = 8,
  ST_COLGATHER = 9,
  ST_DELAY = 10,
  ST_LOC = 11,
  ST_ROWS_ADD = 12,     // adjoint solves: rows of a child's update into its parent
  ST_ROWS_GATHER = 13,  // adjoint solves: a child's boundary rows from its parent
};

struct Step {
  int32_t kind;
  int32_t begin, count;  // descriptor range in the table of the step's kind
  int32_t max_dim;       // largest matrix edge in the step (launch shaping)
};

struct TileRef { int32_t desc, tm, tn, pad; };
// tiles of one GEMM step and its kernel: 0 large tile, 1 small tile, 2 tensor cores,
// 3 one CTA per descriptor (small blocks).  Tensor-core steps also own the
// digit-split work items [sfirst, sfirst + scount); their tiles refer to
// TcDesc entries.
struct TileRange { int32_t first, count, kind, sfirst, scount, dim; };  // dim: largest m, n or k of the launch

// Tensor-core products (FP32 pairs): output tiles of TC_M x TC_N, operands
// as TC_DIGITS 8-bit digit planes per real, 16 k per block.  Per energy, the
// scratch of a step holds for every descriptor the planes of op(A)
// [3][kb][rba][TC_DIGITS][TC_M x 16] and of op(B)^T [3][kb][rbb][TC_DIGITS][TC_N x 16]
// (components Re, Im, Re + Im) and the exponents of the rows of op(A) and
// columns of op(B).
constexpr int TC_M = 128, TC_N = 64, TC_DIGITS = 7;
constexpr int64_t TC_PLANE_A = int64_t(TC_M) * 16, TC_PLANE_B = int64_t(TC_N) * 16;  // bytes
struct TcDesc {
  int64_t dig_a, dig_b;  // byte offsets of the digit planes in the per-energy scratch
  int64_t exp_a, exp_b;  // int32 offsets of the exponents (rba * TC_M and rbb * TC_N entries)
  int32_t desc;          // GEMM descriptor
  int32_t kb, rba, rbb;  // 16-k blocks, TC_M-row blocks of op(A), TC_N-column blocks of op(B)
};
// 32 rows of op(A) (side 0) or columns of op(B) (side 1) to split
struct TcSplit { int32_t tcd, side, r0, pad; };

}  // namespace ndgf

struct nd_plan {
  int32_t n = 0, nnz = 0;
  std::vector<int32_t> rowptr, colind;
  std::vector<int32_t> csr_T;      // CSR index of the transposed entry (colind[q], row of q)
  int32_t n_contacts = 0;
  std::vector<int32_t> contact_ptr, contact_idx;
  std::vector<ndgf::Cluster> cl;  // postorder
  int32_t n_levels = 0, n_roots = 0, max_n = 0, max_b = 0;
  std::vector<int32_t> owner, pos; // owning cluster and front row, per site and per virtual id
  int32_t delay = 0;               // nd_opts.delay
  int32_t n_virtual = 0;           // virtual unknowns (delayed rows), ids n .. n + n_virtual - 1
  int64_t n_unk = 0;               // front rows of all clusters (n + n_virtual)
  int64_t arena_elems = 0;         // complex elements per energy (base regions)
  int64_t ext_elems[2] = {0, 0};   // extra elements of the G^< blocks, per variant
  int64_t sigma_elems = 0;         // sum_c m_c^2
  int64_t root_scratch_elems = 0;  // complex128 scratch of the root blocks per energy (single-precision paths)
  int64_t adj_elems = 0;           // per-energy elements of the adjoint blocks
  int32_t adj_cols = 0;            // M: number of contact sites
  double flops_factor = 0, flops_green_r = 0, flops_green_lesser = 0;

  // device-independent descriptor tables (uploaded by nd_fact_create)
  std::vector<int32_t> sites;        // concatenated front-row lists (caller ids; virtual ids >= n)
  std::vector<int32_t> unk_q, unk_r; // per unknown: cluster and front row (static order)
  std::vector<int32_t> maps;         // concatenated child maps
  std::vector<int32_t> ent_dst;      // assembly: destination offset within off_F region
  std::vector<int32_t> ent_src;      // assembly: CSR value index
  std::vector<ndgf::AssembleDesc> asm_desc;
  std::vector<ndgf::InvDesc> inv_desc;
  std::vector<ndgf::GemmDesc> gemm_desc;
  std::vector<ndgf::ScatterDesc> scat_desc;
  std::vector<ndgf::GatherDesc> gath_desc;
  std::vector<ndgf::DiagDesc> diag_g, diag_p[2];
  std::vector<ndgf::NPhDesc> nph_desc;
  std::vector<ndgf::ZeroDesc> zero_desc;
  std::vector<ndgf::AncGatherDesc> anc_desc;
  std::vector<ndgf::RowScatterDesc> rows_desc;
  std::vector<ndgf::ColGatherDesc> colg_desc;
  std::vector<ndgf::DelayDesc> delay_desc;
  std::vector<ndgf::LocDesc> loc_desc;
  std::vector<int32_t> site_ids;   // B lists as unknown ids (sb of the owner + front row)
  std::vector<int32_t> anc_q, anc_r; // ancestor columns: (cluster, eliminated row)
  std::vector<int32_t> cmaps;      // column maps of ColGatherDesc
  // per-cluster tables for the G lookup of AncGatherDesc (variant v = 0, 1)
  std::vector<int32_t> cl_n, cl_A, cl_ldG;
  std::vector<int64_t> cl_offG, cl_offGX[2], cl_offP[2];
  // per contact: cluster holding its sites, first front row there, offset of
  // its block in the packed Sigma arrays (elements)
  std::vector<int32_t> contact_cluster, contact_row;
  std::vector<int64_t> contact_soff;
  std::vector<ndgf::ZeroDesc> psi_desc;  // Psi regions (growth indicator)
  // residual certificate: for site j, terms [cert_ptr[j], cert_ptr[j+1]) of
  // sum_k A_jk X_kj, each with the neighbour site cert_nb and the coefficient
  // source cert_coef (CSR index >= 0, or -1 - packed Sigma index); where X_kj
  // is stored is found at run time from cert_slot (static slot of every site),
  // cert_cl and the sorted boundary slots cert_bslot / cert_bidx
  std::vector<int32_t> cert_ptr, cert_nb, cert_coef, cert_slot, cert_bslot, cert_bidx;
  std::vector<ndgf::CertCluster> cert_cl;
  // launch schedules: the fold (S1-S3), the G^r extraction (S4) and the
  // G^< / G^> steps (S5-S8) without (0) or with (1) a phonon self-energy
  std::vector<ndgf::Step> sched_factor, sched_green, sched_lesser[2];
};

namespace ndgf {
void build_schedules(nd_plan* p);
}  // namespace ndgf
