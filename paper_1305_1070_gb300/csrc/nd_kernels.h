// Launch wrappers of the device kernels (nd_kernels.cu).  Internal.
#pragma once

#include <cuda_runtime.h>

#include "nd_internal.h"

namespace ndgf {

// Workspace view handed to every launch: per-energy base = arena + e * se,
// auxiliary per-energy base = aux + e * sa (elements of the storage type).
struct Work {
  void* arena;
  int64_t se;
  const void* aux;
  int64_t sa;
  int n_e;
};

// Per-energy row tables of the delayed pivots, [n_e][n_unk] each (all NULL
// when the plan has no delayed rows: then every front row keeps its static
// position and site).
//   iperm: position of each static front row in its cluster's reordered front
//   rsite: caller site of each row of a cluster's front in its current order
//   locq, locr: cluster and eliminated row where each unknown ends up
struct DelayTabs {
  int32_t *iperm, *rsite, *locq, *locr;
  int64_t n_unk;
};

// Per-unknown and per-cluster tables read by the ancestor gather.
struct AncTables {
  const int32_t *site_ids, *unk_q, *unk_r, *anc_q, *anc_r, *cl_n, *cl_A, *cl_ldG;
  const int64_t *cl_offG, *cl_offGX;
};

struct CertArgs {
  int n;
  const int32_t *cptr, *nb, *coef;   // terms of site j: [cptr[j], cptr[j+1]), neighbour site, coefficient source
  const int32_t *slot, *bslot, *bidx; // static slot of every site; sorted boundary slots per cluster
  const int32_t *unk_q, *unk_r;      // static cluster and front row of every slot
  const CertCluster* cl;
  const double *H, *sr, *sl, *ph_r, *ph_l, *energies;
  int64_t sstride;
  double eta;
  int lesser;
  double* cert;  // [n_e][8]
  const ZeroDesc* psi;
  int n_psi;
};

// Contacts passed by value to a kernel (nd_sigma_lesser_fermi in groups of
// this size, the adjoint contraction).
static constexpr int MAX_CONTACTS = 8;
struct ContactTable {
  int32_t n;
  int32_t m[MAX_CONTACTS];
  int64_t off[MAX_CONTACTS];
  double mu[MAX_CONTACTS];
};

template <typename T>
struct Kern {
  static void assemble(const Work& w, const AssembleDesc* d, int count, const int32_t* ent_dst,
                       const int32_t* ent_src, const int32_t* sites, const double* H, const double* energies,
                       double eta, const double* sigma_r, int64_t sigma_stride, const double* ph_r, int n,
                       const DelayTabs& dt, cudaStream_t s);
  static void delay(const Work& w, const DelayDesc* d, int count, int max_nf, const DelayTabs& dt, cudaStream_t s);
  static void inverse(const Work& w, const InvDesc* d, int count, int max_n, double* fp64_scratch,
                      int64_t scratch_stride, int* n_singular, cudaStream_t s);
  // variant 0 large tile, 1 small tile, 2 extra large tile (gemm_tile / gemm_tile_n: its edges)
  static void gemm(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, int variant, cudaStream_t s);
  // one CTA per descriptor (launches whose blocks have every edge <= 96)
  static void gemm_direct(const Work& w, const GemmDesc* d, const TileRef* tiles, int n_tiles, cudaStream_t s);
  static void scatter(const Work& w, const ScatterDesc* d, int count, const int32_t* maps, cudaStream_t s);
  static void gather(const Work& w, const GatherDesc* d, int count, const int32_t* maps, bool skew,
                     const DelayTabs& dt, cudaStream_t s);
  static void zero(const Work& w, const ZeroDesc* d, int count, cudaStream_t s);
  static void nph(const Work& w, const NPhDesc* d, int count, const int32_t* sites, const double* ph_l,
                  const double* ph_g, int n, const DelayTabs& dt, cudaStream_t s);
  static void gather_anc(const Work& w, const AncGatherDesc* d, int count, const AncTables& t, const DelayTabs& dt,
                         cudaStream_t s);
  static void scatter_rows(const Work& w, const RowScatterDesc* d, int count, const int32_t* maps,
                           const DelayTabs& dt, cudaStream_t s);
  static void colgather(const Work& w, const ColGatherDesc* d, int count, const int32_t* cmaps, const AncTables& t,
                        const DelayTabs& dt, cudaStream_t s);
  static void certificate(const Work& w, const CertArgs& a, const DelayTabs& dt, cudaStream_t s);
  static void selected(const Work& w, const CertArgs& a, const DelayTabs& dt, const int32_t* x, const int32_t* y,
                       int count, int lesser, double* Gr, double* Gl, double* Gg, int* n_missing, cudaStream_t s);
  static void diag_out(const Work& w, const DiagDesc* d, int count, const int32_t* sites, double* out, int n,
                       const DelayTabs& dt, cudaStream_t s);
  static void convert_aux(const Work& w, const double* lesser, const double* greater, int64_t sigma_elems,
                          cudaStream_t s);
  static void rows(const Work& w, const RowsDesc* d, int count, const int32_t* maps, int M, bool gather,
                   const DelayTabs& dt, cudaStream_t s);
  static void adj_ones(const Work& w, const int64_t* offs, int count, cudaStream_t s);
  static void zero_range(const Work& w, int64_t off, int64_t count, cudaStream_t s);
  static void adj_mid(const Work& w, const AdjDesc* d, int count, int M, const double* c, const int32_t* sites,
                      const DelayTabs& dt, int mode, cudaStream_t s);
  static void adj_contract(const Work& w, const AdjDesc* d, int count, int M, const ContactTable& ct,
                           const double* sl, int64_t sstride, const int32_t* sites, const DelayTabs& dt, double* out,
                           int n, int forward, cudaStream_t s);
  static void current(const Work& w, int64_t offPl, int64_t offPg, int ld, int row0, int m, const double* sl,
                      const double* sg, int64_t sstride, int64_t soff, double* out, double* out_im, cudaStream_t s);
  static int gemm_tile(int variant);
  static int gemm_tile_n(int variant);
};

// FP32-pair GEMM of one schedule step on the tensor cores (nd_gemm_tc.cu):
// exact BF16 digit products (tcgen05), TC_M x TC_N tiles.  gemm_tc_scratch
// fills the layout fields of t for descriptor g placed at byte offset off of
// the per-energy scratch and returns the offset after it.
int64_t gemm_tc_scratch(const GemmDesc& g, TcDesc& t, int64_t off);
void launch_gemm_tc(const Work& w, const GemmDesc* d, const TcDesc* tcd, const TcSplit* splits, int n_splits,
                    const TileRef* tiles, int n_tiles, unsigned char* scratch, int64_t ss, int* timeout,
                    int64_t wait_polls, cudaStream_t s);

// Sets the function attributes (dynamic shared memory limits) of every kernel
// once; called before any launch can be recorded into a graph.
void prepare_kernels();
void prepare_gemm_tc();

// Final positions of the unknowns after the delayed pivots (one tree level).
void launch_loc(const LocDesc* d, int count, int n_e, const DelayTabs& dt, cudaStream_t s);

// Per-energy complex128 workspace of launch_lead_decimation, in elements.
size_t lead_decimation_work_elems(int m, int m_c);
void launch_lead_decimation(const double* H00, const double* H01, const double* tau, int m, int m_c,
                            const double* energies, int n_e, double eta, double scale, double tol, int max_iter,
                            double* out, int64_t stride, int64_t offset, double* work, int* status, cudaStream_t s);
void launch_lead_modes(const double* U, const double* eps, int m, double hop, const double* energies, int n_e,
                       double eta, double* out, int64_t stride, int64_t offset, cudaStream_t s);
void launch_sigma_lesser(const double* sigma_r, int n_e, const ContactTable& ct, double kT, const double* energies,
                         int64_t stride, double* lesser, double* greater, cudaStream_t s);
void launch_density(const double* X, const double* w, int n_e, int n, double scale, int accumulate, double* out,
                    cudaStream_t s);
void launch_phonon(int n, int n_e, double gamma, double mu, double kT, const double* energies, double* r,
                   double* l, double* g, cudaStream_t s);
void launch_phonon_scba(int n, int n_e, double D, double mix, const double* Gr, const double* Gl, const double* Gg,
                        double* r, double* l, double* g, double* stats, cudaStream_t s);

}  // namespace ndgf
