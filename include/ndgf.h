/*
 * ndgf.h -- C ABI of the GB300 nested-dissection NEGF diagonal solver.
 *
 * The library computes, for a batch of energies E_e, the diagonals of the
 * retarded Green's function G^r = A^{-1} and of the correlation functions
 * G^< = G^r Sigma^< (G^r)^dagger and G^> = G^r Sigma^> (G^r)^dagger, with
 *     A(E) = (E + i eta) I - H - Sigma^r_L - Sigma^r_R - Sigma^r_ph
 * (Hetmaniuk, Zhao, Anantram, arXiv 1305.1070, Eq. (1)-(2)), by a
 * nested-dissection cluster tree (Sec. 3.2): a bottom-up block LDL^T "fold"
 * with separator Schur complements, the root inversion, a top-down selected
 * inversion ("extract") of G^r, and the four-step extension for G^< and G^>.
 *
 * Conventions shared by every entry point
 *  - Complex arrays are interleaved (re, im) doubles, row major, energy-major:
 *    element (e, i, j) of a batch of m x m blocks is at 2*((e*m + i)*m + j).
 *  - Site indices are the caller's 0-based indices of the graph ("caller
 *    order"); all outputs are returned in caller order.
 *  - Ownership: the caller owns every buffer it passes; the library never
 *    frees or retains them beyond the call (stream-ordered calls read/write
 *    them until the work on the stream completes).  Opaque handles own their
 *    internal host and device memory and are released by the *_destroy calls.
 *  - Pointers to per-energy arrays of nd_factor / nd_diag_green may be device
 *    pointers or host pointers; host data is staged through the handle's
 *    device buffers on the given stream (host memory must then stay valid
 *    until the stream is synchronised).  Every other array argument is
 *    documented as host or device.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream); all
 *    device work of a call is ordered on it.  Calls on one handle must not run
 *    concurrently.
 *  - Errors: every entry point returns an nd_status; no exception crosses the
 *    ABI and no device trap is used.  nd_last_error() returns a thread-local
 *    message describing the last non-OK status of the calling thread.
 */
#ifndef NDGF_H
#define NDGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ND_OK = 0,
  ND_ERR_INVALID_ARG = 1,        /* bad size, NULL, out-of-range index          */
  ND_ERR_NOT_SYMMETRIC = 2,      /* pattern, H values or Sigma^r block not symmetric */
  ND_ERR_SINGULAR = 3,           /* exactly singular pivot in a cluster block   */
  ND_ERR_NOT_SKEW_HERMITIAN = 4, /* Sigma^< / Sigma^> block not skew-Hermitian  */
  ND_ERR_OOM = 5,                /* device or host allocation failed            */
  ND_ERR_CUDA = 6,               /* a CUDA runtime call failed                  */
  ND_ERR_TIMEOUT = 7,            /* a bounded device wait gave up               */
  ND_ERR_UNSUPPORTED = 8         /* valid request the library does not handle   */
} nd_status;

/* Arithmetic of the cluster blocks and products: complex128; complex64
 * (FP32, with complex128 root inversion); or complex numbers whose parts are
 * unevaluated sums of two FP32 numbers ("double-float", ~48-bit significand,
 * computed on the FP32 pipe with error-free transforms, complex128 root). */
typedef enum { ND_PREC_FP64 = 0, ND_PREC_MIXED = 1, ND_PREC_FP32X2 = 2 } nd_precision;

/* nd_fact_create flags.  ND_FACT_PHONON: reserve the G^< workspace of every
 * cluster so that nd_diag_green accepts a phonon Sigma^< / Sigma^> (without it
 * only the clusters on the path from a contact to the root carry that
 * workspace). */
#define ND_FACT_PHONON 1
/* GEMM tile size of the batched Schur products.  By default every launch
 * (one tree level of one product) takes the large or the small tile,
 * whichever covers its matrices with less padded work, the small tile being
 * charged a fixed per-flop overhead; these flags force one size
 * (complex128 / FP32 pairs: 32x32 or 16x16; complex64: 64x64 or 32x32). */
#define ND_FACT_TILE_LARGE 2
#define ND_FACT_TILE_SMALL 4
/* Force the extra large tile (64 x 64 with 4 x 4 outputs per thread; 128 x 64
 * for complex64) on every GEMM launch that is not on the tensor cores. */
#define ND_FACT_TILE_XL 128
/* FP32-pair precision only: the Schur products may instead run on the tensor
 * cores (tcgen05), as exact products of 8-bit digits of a 54-bit fixed-point
 * form of each row and column (BF16 in, exact FP32 group sums in tensor
 * memory, FP32-pair accumulation; same accuracy class).  By default the
 * launches whose largest block edge exceeds 192 take them, unless their digit
 * planes would exceed 512 MiB per energy or 64 GiB for all max_ne energies of
 * the handle; ND_FACT_GEMM_TC forces them for
 * every GEMM launch, ND_FACT_GEMM_ALU never uses them.  Their waits are
 * bounded: a wait that gives up makes nd_fact_status return ND_ERR_TIMEOUT. */
#define ND_FACT_GEMM_TC 8
#define ND_FACT_GEMM_ALU 16
/* Reserve the workspace of nd_density_gradient (M right-hand sides per
 * cluster, M = number of contact sites). */
#define ND_FACT_ADJOINT 32
/* Record the device work of nd_factor and of nd_diag_green (a few hundred
 * launches each) once per distinct call shape (energy count, which inputs and
 * outputs are given, eta) into a CUDA graph, and replay it with one
 * cudaGraphLaunch on the caller's stream afterwards.  The input staging copies
 * and the output copies stay outside the graph (outputs always go through the
 * handle's buffers then), so the caller's pointers may change between calls.
 * Not used while the launch profiler is on. */
#define ND_FACT_GRAPH 64

/* Sparsity pattern of H plus the contact site sets (host arrays).
 * rowptr[n+1], colind[nnz]: CSR pattern, 0-based, must be structurally
 * symmetric; the diagonal may be present or absent.  Contact c owns sites
 * contact_idx[contact_ptr[c] .. contact_ptr[c+1]); the contact self-energy
 * block Sigma_c is dense over those sites in that order (paper Sec. 2: the
 * leads fold into dense first/last-layer blocks).  coords[n][coord_dim]
 * (optional, NULL allowed) are site positions used to choose separators. */
typedef struct nd_graph {
  int32_t n;
  const int32_t* rowptr;
  const int32_t* colind;
  int32_t n_contacts;
  const int32_t* contact_ptr;
  const int32_t* contact_idx;
  int32_t coord_dim;
  const double* coords;
} nd_graph;

/* Options of nd_analyze.  leaf_size: maximal number of sites of a leaf
 * cluster (0 = default 64); a contact set is never split, so a contact leaf
 * may be larger.  split_permille: position of each cut as a quantile of the
 * sites' keys, in 1/1000 (0 = default 500, the median); other values give a
 * different tree over the same graph.  slab: when > 0, every cut across the
 * first coordinate axis (transport) is placed `slab` distinct coordinate
 * values below the high end instead of at the quantile, so the tree is a
 * chain of separators, each holding the low-side contact in its subtree, with
 * slabs of `slab` layers dissected below them (paper Sec. 3.2, Fig. 6 is the
 * case slab = 1 without the inner dissection).
 * delay (0..8): delayed pivots, an extension of the paper's elimination.
 * Every cluster that is not a root and holds no contact site leaves `delay`
 * of its front rows uneliminated and hands them to its parent as extra
 * interior unknowns.  The rows are chosen per energy as the largest diagonal
 * entries of the front's inverse, one at a time, updating the inverse after
 * each choice (complex64 selection).  This keeps the fold bounded where an
 * isolated cluster is close to resonance, which the paper's scheme without
 * pivoting across clusters is not.  The result is the same matrix function;
 * only the elimination order differs per energy.  delay > 0 adds an unknown
 * id range n .. n + n_virtual - 1 to the cluster site lists
 * (nd_plan_cluster_sites). */
typedef struct nd_opts {
  int32_t leaf_size;
  int32_t split_permille;
  int32_t slab;
  int32_t delay;        /* delayed pivots per cluster, 0..8 (0 = none) */
  int32_t reserved[4];
} nd_opts;

typedef struct nd_plan nd_plan; /* symbolic analysis (host + device copy)      */
typedef struct nd_fact nd_fact; /* per-energy numeric workspace (device)       */
typedef struct nd_lead nd_lead; /* semi-infinite lead description (host+device) */

/* Summary of a plan.  Flop counts are real floating-point operations per
 * energy with 8 per complex multiply-add, for the fold (factor), the G^r
 * extraction, and the G^< + G^> part (both right-hand sides). */
typedef struct nd_plan_info {
  int32_t n, nnz, n_clusters, n_levels;
  int32_t max_n, max_b, n_contacts, n_roots;
  double flops_factor, flops_green_r, flops_green_lesser;
  double arena_bytes_fp64, arena_bytes_fp32; /* device workspace per energy */
} nd_plan_info;

/* ---- S0: ordering (paper Sec. 3.2 "Comments on the system partition") ------
 * Nested dissection with width-1 separators: recursive bisection of the site
 * set (coordinate median when coords are given, else breadth-first level
 * structure), separator = the sites of one side that touch the other side;
 * a contact set that a cut would split is peeled off as a leaf with its
 * neighbourhood as separator, so Sigma_c and Sigma^<_c stay inside one
 * cluster (paper Fig. 8).  Clusters on one level never couple.  Host only:
 * callable without a GPU.  Errors: ND_ERR_INVALID_ARG (sizes, indices),
 * ND_ERR_NOT_SYMMETRIC (pattern). */
nd_status nd_analyze(const nd_graph* graph, const nd_opts* opts, nd_plan** out);
nd_status nd_plan_query(const nd_plan* plan, nd_plan_info* out);
/* Per-cluster tree arrays (host, each of length n_clusters, any may be NULL):
 * level (1 = leaf), parent (-1 = root), n_i (front rows: interior size, plus
 * the rows delayed from this cluster when nd_opts.delay > 0), b_i (boundary
 * size, counting the cluster's own delayed rows first).  cluster_of_site[n]
 * (may be NULL): owning cluster of each site. */
nd_status nd_plan_tree(const nd_plan* plan, int32_t* level, int32_t* parent, int32_t* n_i,
                       int32_t* b_i, int32_t* cluster_of_site);
/* Sites of cluster c: interior set I_c (n_c entries) then boundary set B_c
 * (b_c entries), caller order, written to a host array of n_c + b_c ints. */
nd_status nd_plan_cluster_sites(const nd_plan* plan, int32_t c, int32_t* sites);
void nd_plan_destroy(nd_plan* plan);

/* ---- numeric workspace -----------------------------------------------------
 * Allocates device memory for up to max_ne energies at the given precision
 * (nd_precision).  flags: ND_FACT_*.
 * The plan must outlive the handle.  Errors: ND_ERR_OOM, ND_ERR_CUDA,
 * ND_ERR_INVALID_ARG; ND_ERR_UNSUPPORTED for a cluster of more than 8192
 * interior or 32768 boundary sites, or more than two contacts in one cluster.
 * The kernels put the energy on the grid's y dimension, so max_ne must not
 * exceed 65535 (a larger value makes the launches fail with ND_ERR_CUDA; the
 * Python binding refuses it with ND_ERR_UNSUPPORTED before allocating). */
nd_status nd_fact_create(const nd_plan* plan, int32_t max_ne, int32_t precision, int32_t flags, nd_fact** out);
void nd_fact_destroy(nd_fact* fact);

/* ---- S1 + S2 + S3: assemble and fold (paper Sec. 3.2, "folding", root) -----
 * H_values[nnz]          : values of H aligned with the graph's colind (real).
 * sigma_r                : [n_e][sum_c m_c^2] complex, contact blocks Sigma^r_c
 *                          (contact order, each m_c x m_c row major); the
 *                          blocks must be complex symmetric.
 * sigma_ph_r             : [n_e][n] complex diagonal Sigma^r_ph, or NULL.
 * energies               : [n_e] real.
 * eta                    : positive broadening added to the device diagonal
 *                          (eta <= 0 or not finite: ND_ERR_INVALID_ARG; with
 *                          eta = 0 an interior block E - H_ii can be exactly
 *                          singular).
 * Folds every cluster level by level (Psi_i = -A_ii^{-1} A_{i,B}, Schur update
 * of the parent front) and inverts the root.  The elimination relies on
 * A = A^T (paper Sec. 3.1, LDL^T), so H must have symmetric values and every
 * Sigma^r_c block must be complex symmetric, within the relative tolerance of
 * nd_check_factor_inputs: host arrays are checked before any device work
 * (ND_ERR_NOT_SYMMETRIC from this call), device arrays by a kernel on the
 * stream (ND_ERR_NOT_SYMMETRIC from the next nd_fact_status; the results are
 * then invalid).  Errors: ND_ERR_INVALID_ARG, ND_ERR_NOT_SYMMETRIC,
 * ND_ERR_CUDA; ND_ERR_SINGULAR is reported by nd_fact_status after the stream
 * is synchronised (no device trap). */
nd_status nd_factor(nd_fact* fact, const double* H_values, const double* sigma_r,
                    const double* sigma_ph_r, const double* energies, int32_t n_e, double eta,
                    void* stream);

/* ---- S4..S8 + S10: selected inversion (paper Sec. 3.2, G^r and G^< steps) --
 * sigma_lesser, sigma_greater : [n_e][sum_c m_c^2] complex contact blocks of
 *                               Sigma^< and Sigma^> (skew-Hermitian), or NULL.
 * ph_lesser, ph_greater       : [n_e][n] complex diagonals, or NULL.
 * Gr, Gl, Gg                  : [n_e][n] complex outputs (diag G^r, G^<, G^>)
 *                               in caller order; NULL skips that output (Gl
 *                               and Gg need the matching Sigma terms).
 * Uses the factorization of the last nd_factor call on this handle.  The
 * Sigma^< / Sigma^> inputs must be skew-Hermitian (paper Sec. 3.1, Eq. (5)-(6):
 * the extraction sets P_BI = -(P_IB)^dagger), within the tolerance of
 * nd_check_lesser_inputs: host arrays are checked before any device work
 * (ND_ERR_NOT_SKEW_HERMITIAN from this call), device arrays on the stream
 * (ND_ERR_NOT_SKEW_HERMITIAN from the next nd_fact_status). */
nd_status nd_diag_green(nd_fact* fact, const double* sigma_lesser, const double* sigma_greater,
                        const double* ph_lesser, const double* ph_greater, double* Gr, double* Gl,
                        double* Gg, void* stream);

/* ---- S9: accuracy certificate ---------------------------------------------
 * For the last nd_factor + nd_diag_green of the handle, in FP64 from the
 * stored selected entries, per energy e and over all sites j:
 *   cert[e][0] = max_j |(A G^r)_jj - 1|,           cert[e][1] = max_j |G^r_jj|,
 *   cert[e][2] = max_j |(A G^<)_jj - (Sigma^< G^a)_jj|, cert[e][3] = max_j |G^<_jj|
 * (paper Eq. (1): A G^r = I and A G^< = Sigma^< (G^r)^dagger; every nonzero
 * A_jk has its G_kj among the entries the selected inversion stores, Sec. 3.2,
 * also with delayed pivots, where the entry's place is found per energy).
 *   cert[e][4] = max over clusters of max |Psi_i| (Psi_i = -A_ii^{-1} A_iB), the
 *                growth of the fold: the extraction multiplies rounding errors
 *                of G_BB by Psi_i, so large values flag energies whose diagonal
 *                carries amplified rounding;
 *   cert[e][5] = 1 if a stored entry could not be located (an internal
 *                inconsistency of the plan; never expected), else 0;
 *   cert[e][6] = max_j |(A G^r)_jj - 1| / max_j (sum_k |A_jk| |G_kj|),
 *   cert[e][7] = max_j |(A G^< - Sigma^< G^a)_jj| / max_j (sum_k |A_jk| |G^<_kj|
 *                + sum_k |Sigma^<_jk| |G_jk|): the residuals relative to the
 *                magnitude of their terms (normwise backward errors of the
 *                diagonal, comparable with the unit roundoff of the path:
 *                ~1e-16 complex128, ~1e-13 FP32 pairs, ~1e-6 complex64).
 * A NaN anywhere makes the affected entries +inf.
 * Entries 2 and 3 are 0 when G^< was not computed.  cert: [n_e][8] doubles,
 * host or device.  Stream ordered after the nd_diag_green call.  The residual
 * of the diagonal is the refinement test of the mixed paths: a residual-
 * correction step G + G (I - A G) would need whole rows of G, which the
 * selected inversion does not form, so an energy whose residual is too large
 * is recomputed on the complex128 path instead (the Python driver's
 * certified step does this). */
nd_status nd_certificate(nd_fact* fact, double* cert, void* stream);

/* Selected entries of the last nd_factor + nd_diag_green (paper Sec. 3.2: the
 * selected inversion stores G^(0) on the fill pattern, i.e. G_xy for every
 * pair x, y that A couples, and every pair inside one cluster's front): for
 * count pairs (x[p], y[p]) of caller sites, for every energy e,
 *   Gr[e][p] = G^r_xy, Gl[e][p] = G^<_xy, Gg[e][p] = G^>_xy
 * ([n_e][count] complex, device; any may be NULL; Gl / Gg need a preceding
 * nd_diag_green that computed G^< or G^>).  Bond currents
 * J_xy(E) ~ Re(H_xy G^<_yx) and the S9 residual are built from these.  A pair
 * whose entry is not stored (not coupled, or out of range) gets NaN and is
 * counted in *n_missing (device int32, cleared by the call).  x, y: device
 * int32 [count].  Errors: ND_ERR_INVALID_ARG. */
nd_status nd_selected_entries(nd_fact* fact, const int32_t* x, const int32_t* y, int32_t count, double* Gr,
                              double* Gl, double* Gg, int32_t* n_missing, void* stream);

/* Adjoint of the density (an extension: the paper computes the density
 * only; its Sec. 1 motivates self-consistent device simulation): for every energy of the last nd_factor / nd_diag_green pair
 * and every site k,
 *     t_k(E) = sum_{a,b in contacts} Sigma^<_ab conj(U_kb) conj(Z_ka),
 *     U = G^r[:, contact sites],  Z = G^r diag(c) conj(U),
 * so that for L = sum_j c_j n_j with n_j = (1/pi) sum_E w_E Im G^<_jj(E) and
 * H_kk = H0_kk + V_k (dA/dV_k = -e_k e_k^T):
 *     dL/dV_k = (2/pi) sum_E w_E Im t_k(E)       (nd_density with scale 2/pi).
 * U and Z come from two solves with the stored factorization (upward sweep
 * RB += Psi^T XI, downward XS = A_ii^{-1} XI + Psi XB), in the workspace's
 * precision.  c: [n] real weights (host or device, caller order);
 * t_out: device [n_e][n] complex.  Needs a workspace created with
 * ND_FACT_ADJOINT, a preceding nd_diag_green given Sigma^<, no phonon
 * Sigma^< (its support is every site) and at most 8 contacts.
 * Errors: ND_ERR_INVALID_ARG, ND_ERR_UNSUPPORTED. */
nd_status nd_density_gradient(nd_fact* fact, const double* c, double* t_out, void* stream);

/* Forward (directional) derivative of the density, for Newton steps of the
 * self-consistent loop (an extension of the paper): for a potential change v of
 * the on-site energies (H_kk = H0_kk + V_k), every energy of the last
 * nd_factor / nd_diag_green and every site j,
 *     T_j(E) = sum_{a,b in contacts} W_ja Sigma^<_ab conj(U_jb),
 *     U = G^r[:, contact sites],  W = G^r diag(v) U,
 * so that with n_j = (1/pi) sum_E w_E Im G^<_jj(E):
 *     (dn/dV v)_j = (2/pi) sum_E w_E Im T_j(E)      (nd_density with scale 2/pi)
 * (dG^r = G^r diag(v) G^r and dG^< = dG^r Sigma^< G^a + G^r Sigma^< dG^a, paper
 * Eq. (1)-(2)).  U is solved once per factorization and kept, so later calls
 * on the same factorization (and nd_density_gradient) take one solve each.
 * v: [n] real (host or device, caller order); t_out: device [n_e][n] complex.
 * Same requirements and errors as nd_density_gradient. */
nd_status nd_density_jvp(nd_fact* fact, const double* v, double* t_out, void* stream);

/* ---- Poisson operator of the self-consistent loop (an extension) -------------
 * On an nx (transport) x ny (transverse) grid, site (x, y) = x * ny + y:
 *     (K u)_j = sum_{k neighbour of j} (u_j - u_k),
 * u = 0 on ghost columns x = -1 and x = nx (Dirichlet at the ends, the leads'
 * potential) and no neighbours across the edges y = 0, ny - 1 (Neumann).  K is
 * symmetric positive definite.  nd_poisson_apply: out = K u; nd_poisson_solve:
 * (K + shift I) u = rhs, shift >= 0 (the screened operator of a Newton
 * preconditioner), directly (cosine transform along y, one tridiagonal solve
 * per mode along x, transform back), FP64.  Arrays are device [batch][nx * ny]
 * doubles; work memory grows on demand inside the handle.  The paper motivates
 * the density by Poisson's equation (Sec. 1) but gives no electrostatics.
 * Errors: ND_ERR_INVALID_ARG (sizes, host arrays), ND_ERR_OOM, ND_ERR_CUDA. */
typedef struct nd_poisson nd_poisson;
nd_status nd_poisson_create(int32_t nx, int32_t ny, nd_poisson** out);
nd_status nd_poisson_apply(nd_poisson* poisson, const double* u, double* out, int32_t batch, void* stream);
nd_status nd_poisson_solve(nd_poisson* poisson, double shift, const double* rhs, double* u, int32_t batch,
                           void* stream);
void nd_poisson_destroy(nd_poisson* poisson);

/* Vector operations of the Newton-Krylov iteration (device arrays of n
 * doubles): *out = sum_i x_i y_i (a fixed reduction order, so repeated calls
 * agree bit for bit; out is a device double), y = a x + b y (b = 0
 * overwrites y), and the elementwise product.  Errors: ND_ERR_INVALID_ARG
 * (host arrays, n < 0). */
nd_status nd_vec_dot(const double* x, const double* y, int64_t n, double* out, void* stream);
nd_status nd_vec_axpby(double a, const double* x, double b, double* y, int64_t n, void* stream);
/* y_i = d_i x_i, and y_i = max(0, a x_i) (device arrays of n doubles; y may alias x). */
nd_status nd_vec_mul(const double* d, const double* x, double* y, int64_t n, void* stream);
nd_status nd_vec_scale_pos(double a, const double* x, double* y, int64_t n, void* stream);

/* S10 terminal current spectrum of one contact (Meir-Wingreen; paper Sec. 1,
 * the current is the physical output next to the density):
 *     i_c(E) = Tr[Sigma^<_c(E) G^>_cc(E) - Sigma^>_c(E) G^<_cc(E)]
 * over the contact's own m_c x m_c block, for every energy of the last
 * nd_factor / nd_diag_green pair (which must have been given Sigma^< and
 * Sigma^>).  The terminal current is (2e/h) times the integral over E.
 * current[n_e] receives the real part, current_im[n_e] (may be NULL) the
 * imaginary part, which is zero up to rounding; both host or device.
 * Errors: ND_ERR_INVALID_ARG (contact out of range, no preceding G^</G^>). */
nd_status nd_contact_current(nd_fact* fact, int32_t contact, double* current, double* current_im,
                             void* stream);

/* ---- S10: density epilogue --------------------------------------------------
 * out[j] = (accumulate ? out[j] : 0) + scale * sum_e weights[e] Im X[e][j],
 * X = diag G^< ([n_e][n] complex, caller order).  With trapezoid weights and
 * scale = 2/(2 pi) this is the spin-degenerate electron density per site
 * (paper Sec. 1: the diagonal of G^< is the electron density per unit energy).
 * All arrays are device pointers. */
nd_status nd_density(const double* Gl, const double* weights, int32_t n_e, int32_t n, double scale,
                     int32_t accumulate, double* out, void* stream);

/* The same density epilogue on the handle's last diag G^< (wherever
 * nd_diag_green put it: the caller's device array, or the handle's staging
 * copy when the caller asked for host output), for the n_e energies of the
 * last nd_factor: out[j] = (accumulate ? out[j] : 0) + scale * sum_e
 * weights[e] Im G^<_jj(E_e).  weights [n_e] and out [n] may be host or device
 * arrays (host arrays are copied on the stream; a host out must stay valid
 * until the stream is synchronised).  Errors: ND_ERR_INVALID_ARG (no G^< in
 * the last nd_diag_green). */
nd_status nd_fact_density(nd_fact* fact, const double* weights, double scale, int32_t accumulate, double* out,
                          void* stream);

/* ---- launch profiling ------------------------------------------------------
 * While enabled, every launch of the fold / extraction schedules on the
 * handle's stream is bracketed by CUDA events.  nd_profile(f, enable, stats,
 * max, &count) synchronises the device, writes per-kernel-kind totals of the
 * launches recorded since the previous call (launch count, milliseconds,
 * algorithmic flops: 8 per complex multiply-add, n^3 complex multiply-adds per
 * n x n inverse), clears them and sets the enable state. */
typedef struct nd_kernel_stats {
  char name[24];
  int32_t launches;
  double ms, flops, bytes;
} nd_kernel_stats;
nd_status nd_profile(nd_fact* fact, int32_t enable, nd_kernel_stats* stats, int32_t max_stats, int32_t* n_stats);
/* The launches recorded since profiling was enabled, one entry each, in launch
 * order (without clearing them; nd_profile clears): step kind (the order of
 * nd_profile's names: 0 inverse, 1 gemm (large ALU tile), 2 scatter, ..., 11 loc,
 * 12 gemm_tc (tensor cores), 13 gemm_small, 14 gemm_direct (one CTA per
 * block), 15 gemm_xl (extra large tile)), descriptors in the
 * launch, largest block edge, energies, CUDA-event time (ms) and algorithmic
 * flops.  n_out receives the number recorded (out may be NULL to query it). */
typedef struct nd_launch_stats {
  int32_t kind, count, max_dim, n_e;
  double ms, flops;
} nd_launch_stats;
nd_status nd_profile_launches(nd_fact* fact, nd_launch_stats* out, int32_t max_out, int32_t* n_out);

/* Status of the last factor/diag call (synchronises the handle's stream):
 * n_singular = number of (energy, cluster) pivots that were exactly zero;
 * returns, in this order of precedence, ND_ERR_TIMEOUT when a bounded wait of
 * a tensor-core product gave up, ND_ERR_NOT_SYMMETRIC / ND_ERR_NOT_SKEW_HERMITIAN
 * when the device inputs of the last nd_factor / nd_diag_green failed their
 * check, ND_ERR_SINGULAR when n_singular > 0 (the results are then invalid). */
nd_status nd_fact_status(nd_fact* fact, int32_t* n_singular);

/* ---- kernel autotuner (energy batching: kernel choice per launch) -------------
 * Measures, on the given inputs (those of nd_factor and nd_diag_green, host
 * or device), every candidate kernel of every GEMM launch of the fold and the
 * extraction: the default rules, the large and the small tile, the tensor
 * cores (FP32 pairs), one CTA per block (blocks up to 192) and an extra large
 * tile (64 x 64, 4 x 4 outputs per thread; 128 x 64 for complex64): one pass
 * per candidate with all its launches on it, each after an untimed pass,
 * `reps` timed passes averaged, CUDA events on the stream.  Each launch then takes
 * its fastest kernel for every later call on the handle (the results are
 * the same up to rounding order).  The call runs 6 (reps + 1) factor +
 * diag_green passes and synchronises the stream; the recorded graphs of
 * ND_FACT_GRAPH are dropped.  The adjoint solves keep the default rules.
 * info (may be NULL): summed GEMM milliseconds of one pass with the default
 * rules and with the chosen kernels, GEMM launches tuned, launches whose
 * kernel changed, passes, and the launches per kernel kind (0 large tile,
 * 1 small tile, 2 tensor cores, 3 one CTA per block, 4 extra large tile).  Errors: those of
 * nd_factor / nd_diag_green, ND_ERR_INVALID_ARG (reps < 1). */
typedef struct nd_tune_info {
  double ms_default, ms_tuned;
  int32_t gemm_steps, changed, passes;
  int32_t by_kind[5];
} nd_tune_info;
nd_status nd_autotune(nd_fact* fact, const double* H_values, const double* sigma_r, const double* sigma_ph_r,
                      const double* sigma_lesser, const double* sigma_greater, const double* ph_lesser,
                      const double* ph_greater, const double* energies, int32_t n_e, double eta, int32_t reps,
                      nd_tune_info* info, void* stream);

/* Number of polls after which a wait of the tensor-core products gives up
 * (0 = the default of 2^25, seconds of waiting).  A wait that gives up makes
 * its CTA wait for its own copies and products in flight (always with the
 * default limit), release its tensor memory and skip its output; the next
 * nd_fact_status returns ND_ERR_TIMEOUT.  A small value makes the waits run
 * out on purpose, which tests that path without a device fault; the handle
 * stays usable (the next nd_factor starts clean).  Errors: ND_ERR_INVALID_ARG. */
nd_status nd_fact_set_wait_limit(nd_fact* fact, int64_t polls);

/* The kernel of every step, as nd_autotune chose it (or as nd_fact_set_choice
 * set it; -1 everywhere on a new handle: the default rules), flattened over
 * the schedules in this order: fold, G^r, G^<, phonon G^<, adjoint forward,
 * adjoint backward.  Entries: -1 default rule, 0 large tile, 1 small tile,
 * 2 tensor cores (FP32 pairs only), 3 one CTA per block (blocks up to 192),
 * 4 extra-large tile; a step that is not a GEMM takes -1.  A stored choice
 * applies to any handle of the same plan, precision and flags (one with fewer
 * energies, say), which then runs the same kernels with the same results.
 * nd_fact_get_choice writes min(count, max) entries (choice may be NULL) and
 * the count to *n; nd_fact_set_choice takes exactly count entries and rebuilds
 * the launch tables.  No counterpart in the paper (an implementation control,
 * like the tuner).  Errors: ND_ERR_INVALID_ARG (count, a value out of range or
 * not allowed on its step; max below the count), ND_ERR_OOM. */
nd_status nd_fact_get_choice(nd_fact* fact, int8_t* choice, int32_t max, int32_t* n);
nd_status nd_fact_set_choice(nd_fact* fact, const int8_t* choice, int32_t n);

/* ---- S1a: contact self-energies (paper Sec. 2) ----------------------------
 * A lead is a semi-infinite chain of principal layers with on-site block H00
 * (m x m real symmetric), hopping H01 (m x m) from a layer to the next one
 * away from the device, attached to the m_c contact sites by tau (m_c x m):
 *     Sigma^r(E) = tau g_s(E) tau^T,  g_s = (z - H00 - H01 g_s H01^T)^{-1},
 *     z = E + i eta.   All three arrays are host, row major.
 * When H01 = -h I and tau = -h I the lead is diagonalised once on the host
 * (transverse modes) and Sigma^r = U diag(h lambda_n) U^T with lambda_n the
 * decaying root of lambda^2 - ((z - eps_n)/h) lambda + 1 = 0.  Any other lead
 * uses the renormalisation-decimation of Lopez Sancho, Lopez Sancho and Rubio
 * (J. Phys. F 15, 851 (1985)) on the device in complex128, one CTA per
 * energy, at most 100 doubling steps, stopping when the effective couplings
 * fall below 1e-14 * max(1, |H00|, |H01|).  The lead copies H00, H01, tau;
 * the caller keeps ownership of its arrays.  Errors: ND_ERR_INVALID_ARG,
 * ND_ERR_NOT_SYMMETRIC (H00), ND_ERR_OOM. */
nd_status nd_lead_create(int32_t m, int32_t m_c, const double* H00, const double* H01,
                         const double* tau, nd_lead** out);
/* Writes Sigma^r of every energy into sigma_out (device, complex): block of
 * energy e starts at complex element e*stride + offset (m_c x m_c row major).
 * energies: device [n_e]. */
nd_status nd_lead_sigma(nd_lead* lead, const double* energies, int32_t n_e, double eta,
                        double* sigma_out, int64_t stride, int64_t offset, void* stream);
/* Decimation leads only: number of energies that had not converged within the
 * step limit and number of exactly singular pivots met, accumulated over the
 * nd_lead_sigma calls since the previous nd_lead_status (then reset).
 * Synchronises the stream of the last nd_lead_sigma call.  Returns
 * ND_ERR_SINGULAR when either count is non-zero; always ND_OK and zeros for a
 * transverse-mode lead. */
nd_status nd_lead_status(nd_lead* lead, int32_t* n_unconverged, int32_t* n_singular);
void nd_lead_destroy(nd_lead* lead);

/* Lesser/greater contact self-energies from the retarded ones (device arrays,
 * packed like nd_factor's sigma_r): Gamma_c = i (Sigma_c - Sigma_c^dagger),
 * Sigma^<_c = i f_c Gamma_c, Sigma^>_c = -i (1 - f_c) Gamma_c with the Fermi
 * function f_c = 1/(1 + exp((E - mu_c)/kT)).  m_c, mu: host [n_contacts]; any
 * number of contacts (a batch of devices in one graph has two per device). */
nd_status nd_sigma_lesser_fermi(const double* sigma_r, int32_t n_e, int32_t n_contacts,
                                const int32_t* m_c, const double* mu, double kT,
                                const double* energies, double* sigma_lesser,
                                double* sigma_greater, void* stream);

/* Self-consistent Born update of an elastic local phonon (dephasing)
 * self-energy (a model the paper leaves open, Sec. 2; S. Datta, Superlattices
 * Microstruct. 28, 253 (2000)): with the diagonals of the last nd_diag_green
 * call (caller order), Sigma^r_ph,jj <- Sigma + mix (D G^r_jj - Sigma), and
 * likewise Sigma^< from i Im G^< and Sigma^> from i Im G^> (D in eV^2,
 * 0 < mix <= 1; the diagonal of a skew-Hermitian G^< is imaginary, so only the
 * rounding residue of Re G^<_jj is dropped, which keeps Sigma^< skew-Hermitian
 * for the input check of nd_diag_green).  All arrays are device [n_e][n] complex; the phonon arrays are updated in
 * place and are the inputs of the next nd_factor / nd_diag_green.
 * stats (device, 2 doubles) receives max |D G - Sigma| and max |D G| over the
 * three self-energies (their ratio is the relative change of the iteration).
 * Errors: ND_ERR_INVALID_ARG (sizes, NULL, host pointers, D or mix). */
nd_status nd_phonon_scba(int32_t n, int32_t n_e, double D, double mix, const double* Gr,
                         const double* Gl, const double* Gg, double* ph_r, double* ph_lesser,
                         double* ph_greater, double* stats, void* stream);

/* Constant-broadening phonon self-energy on every site (device outputs
 * [n_e][n] complex, any may be NULL): Sigma^r = -i gamma/2,
 * Sigma^< = i f(E; mu) gamma, Sigma^> = -i (1 - f) gamma. */
nd_status nd_phonon_const(int32_t n, int32_t n_e, double gamma, double mu, double kT,
                          const double* energies, double* ph_r, double* ph_lesser,
                          double* ph_greater, void* stream);

/* ---- allocation-free batched inversion (no counterpart in the paper) -------
 * For callers that cannot allocate device memory (a frozen or foreign memory
 * pool, allocation forbidden inside a host framework's callbacks, a
 * fixed-footprint service).  Inverts `batch` complex64 matrices A[b] (device,
 * [batch][n][n] interleaved (re, im) floats, row major) in place: each is
 * copied to complex128, inverted by Gauss-Jordan with partial pivoting, and
 * rounded back.  The complex128 copies live in a fixed file-scope device array
 * of 2^18 complex128 elements (4 MiB) that every GPU loading the library holds
 * until the process exits; batch * n * n must not exceed 2^18 (so n <= 512),
 * else ND_ERR_INVALID_ARG, and A and n_singular must be device arrays (else
 * ND_ERR_INVALID_ARG).  No cudaMalloc/cudaFree is called.
 * n_singular (device int32) receives the number of exactly singular pivots
 * (it is cleared by the call).  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and must be serialised by the caller. */
nd_status nd_invert_c64_noalloc(float* A, int32_t n, int32_t batch, int32_t* n_singular, void* stream);

/* ---- input checks (host arrays; callable without a GPU) ----------------------
 * The checks nd_factor and nd_diag_green apply to their host inputs, on their
 * own.  nd_check_factor_inputs: H_values[nnz] symmetric on the pattern,
 * |H_jk - H_kj| <= 1e-8 max(|H_jk|, |H_kj|), and every contact block of
 * sigma_r ([n_e][sum_c m_c^2] complex, may be NULL when the plan has no
 * contacts) complex symmetric, |S_ab - S_ba| <= 1e-8 max|S| per block and
 * energy (paper Sec. 3.1: the fold is an LDL^T elimination of A = A^T):
 * ND_ERR_NOT_SYMMETRIC.  nd_check_lesser_inputs: every contact block of
 * sigma_lesser / sigma_greater skew-Hermitian, |S_ab + conj(S_ba)| <= 1e-8
 * max|S|, and the phonon diagonals ph_lesser / ph_greater ([n_e][n] complex)
 * purely imaginary, |Re s_j| <= 1e-8 |s_j| (paper Sec. 3.1, Eq. (5)-(6)); any
 * pointer may be NULL: ND_ERR_NOT_SKEW_HERMITIAN.  Non-finite values fail the
 * check.  Errors: ND_ERR_INVALID_ARG (NULL plan or H, n_e < 0). */
nd_status nd_check_factor_inputs(const nd_plan* plan, const double* H_values, const double* sigma_r, int32_t n_e);
nd_status nd_check_lesser_inputs(const nd_plan* plan, const double* sigma_lesser, const double* sigma_greater,
                                 const double* ph_lesser, const double* ph_greater, int32_t n_e);

const char* nd_last_error(void);
const char* nd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NDGF_H */
