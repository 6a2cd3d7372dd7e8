// Host side of the C ABI: numeric workspace, schedule execution and the
// self-energy helpers.  Every device step runs in the kernels of
// nd_kernels.cu; there is no host fallback.

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "nd_arith.cuh"
#include "nd_check.h"
#include "nd_internal.h"
#include "nd_kernels.h"

using namespace ndgf;

namespace {

#define ND_CUDA(call)                                                                                       \
  do {                                                                                                      \
    cudaError_t _e = (call);                                                                                \
    if (_e != cudaSuccess) return fail(ND_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

template <typename V>
nd_status upload(const std::vector<V>& h, V** d) {
  *d = nullptr;
  if (h.empty()) return ND_OK;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(V));
  if (e != cudaSuccess) return fail(ND_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  return ND_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace {
// Per-kind launch timing with CUDA events on the launching stream.
constexpr int PROF_GEMM_TC = 12;  // profiler kind of the tensor-core GEMM launches

struct Profiler {
  bool on = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
    int count = 0, max_dim = 0, n_e = 0;
    const void* tr = nullptr;  // tile ranges of the schedule and index of the step (the tuner's key)
    int si = -1;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void clear() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  ~Profiler() {
    clear();
    for (auto e : pool) cudaEventDestroy(e);
  }
};
}  // namespace

struct nd_fact {
  const nd_plan* plan = nullptr;
  int precision = ND_PREC_FP64;
  int max_ne = 0;
  int n_e = 0;  // energies of the last nd_factor
  size_t esize = 16;
  void* arena = nullptr;
  void* aux = nullptr;
  double* root_scratch = nullptr;
  int64_t root_stride = 0;
  int* d_status = nullptr;
  int* d_inerr = nullptr;  // [0] inputs of nd_factor not symmetric, [1] inputs of nd_diag_green not skew-Hermitian
  int32_t* d_csrT = nullptr;  // CSR transpose index (symmetry check of device H)
  int32_t* d_cm = nullptr;    // contact sizes
  int64_t* d_csoff = nullptr; // contact block offsets in the packed Sigma arrays
  bool has_ph = false;
  // device tables
  int32_t *d_sites = nullptr, *d_maps = nullptr, *d_ent_dst = nullptr, *d_ent_src = nullptr;
  AssembleDesc* d_asm = nullptr;
  InvDesc* d_inv = nullptr;
  GemmDesc* d_gemm = nullptr;
  ScatterDesc* d_scat = nullptr;
  GatherDesc* d_gath = nullptr;
  DiagDesc *d_diag_g = nullptr, *d_diag_p[2] = {nullptr, nullptr};
  NPhDesc* d_nph = nullptr;
  ZeroDesc* d_zero = nullptr;
  AncGatherDesc* d_anc = nullptr;
  RowScatterDesc* d_rows = nullptr;
  ColGatherDesc* d_colg = nullptr;
  DelayDesc* d_delay = nullptr;
  LocDesc* d_loc = nullptr;
  DelayTabs dt{nullptr, nullptr, nullptr, nullptr, 0};  // per-energy row tables (delayed pivots)
  int32_t *d_unk_q = nullptr, *d_unk_r = nullptr, *d_anc_q = nullptr, *d_anc_r = nullptr;
  int32_t *d_site_ids = nullptr, *d_cmaps = nullptr, *d_owner = nullptr, *d_pos = nullptr;
  int32_t *d_cl_n = nullptr, *d_cl_A = nullptr, *d_cl_ldG = nullptr;
  int64_t *d_cl_offG = nullptr, *d_cl_offGX[2] = {nullptr, nullptr};
  int flags = 0;
  int64_t se = 0;  // workspace elements per energy
  // inputs of the last nd_factor / nd_diag_green (staged copies) for nd_certificate
  double eta = 0.0;
  const double *cur_H = nullptr, *cur_sr = nullptr, *cur_ph = nullptr, *cur_E = nullptr;
  const double *cur_sl = nullptr, *cur_sg = nullptr, *cur_pl = nullptr;
  double* d_current = nullptr;  // [max_ne][2]: Re and Im of the last current spectrum
  // adjoint solves (ND_FACT_ADJOINT)
  bool adj = false;
  int64_t adj_base = 0;
  std::vector<Step> sched_adj_fwd, sched_adj_bwd;
  std::vector<TileRange> tr_adj_fwd, tr_adj_bwd;
  std::vector<double> step_flops_adj_fwd, step_flops_adj_bwd;
  RowsDesc* d_rows_adj = nullptr;
  AdjDesc* d_adj_desc = nullptr;
  int n_adj_desc = 0;
  int64_t* d_ones = nullptr;
  int n_ones = 0;
  double* d_cvec = nullptr;
  bool have_lesser = false;
  bool have_green = false;  // an nd_diag_green followed the last nd_factor
  bool adj_u_valid = false;  // the adjoint region holds U = G^r E_C of the current factorization
  const double* last_gl = nullptr;  // device diag G^< of the last nd_diag_green (the caller's array or staging)
  double *d_w = nullptr, *d_dens = nullptr;  // nd_fact_density: weights [max_ne], density [n]
  double* d_cert = nullptr;
  int32_t *d_cert_ptr = nullptr, *d_cert_nb = nullptr, *d_cert_coef = nullptr, *d_cert_slot = nullptr;
  int32_t *d_cert_bslot = nullptr, *d_cert_bidx = nullptr;
  CertCluster* d_cert_cl = nullptr;
  ZeroDesc* d_psi = nullptr;
  Profiler prof;
  std::vector<double> step_flops_factor, step_flops_green, step_flops_lesser[2];  // per step, per energy
  TileRef* d_tiles = nullptr;
  // tensor-core steps (FP32 pairs): layouts, split items, per-energy scratch
  TcDesc* d_tcd = nullptr;
  TcSplit* d_tcsplit = nullptr;
  unsigned char* tc_scratch = nullptr;
  int64_t tc_stride = 0;  // bytes per energy
  int* d_tc_timeout = nullptr;
  int64_t tc_wait_polls = 0;  // polls before a tensor-core wait gives up (0 = the kernel's default)
  // tile range of every GEMM step: index = step index in its schedule
  std::vector<TileRange> tr_factor, tr_green, tr_lesser[2];
  std::vector<GemmDesc> gemm_all;  // the plan's GEMM table plus the adjoint's (host copy)
  bool tuned = false;
  std::array<std::vector<int8_t>, 6> choice;  // kernel per step of each schedule (-1: default rules)
  // staging buffers for host inputs / outputs
  double *st_H = nullptr, *st_sr = nullptr, *st_ph = nullptr, *st_E = nullptr;
  double *st_sl = nullptr, *st_sg = nullptr, *st_pl = nullptr, *st_pg = nullptr;
  double *st_out[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> allocs;

  // ND_FACT_GRAPH: the launch sequence of each (call kind, energy count,
  // inputs present, ...) recorded once into a CUDA graph on a private
  // capture stream and replayed with one cudaGraphLaunch on the caller's stream
  struct GraphEntry {
    uint64_t key[2];
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;

  void clear_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  ~nd_fact() {
    clear_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

nd_status dalloc(nd_fact* f, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return ND_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ND_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  f->allocs.push_back(*p);
  return ND_OK;
}

template <typename V>
nd_status dupload(nd_fact* f, const std::vector<V>& h, V** d) {
  nd_status st = upload(h, d);
  if (*d) f->allocs.push_back(*d);
  return st;
}

// Tile lists of the GEMM steps.  Each step takes the large or the small tile:
// forced by the workspace flags, else the one with less padded work
// sum(tiles * tile area * k), the small tile's work weighted by small_cost
// (its lower reuse per loaded element; measured on the 512 x 128 workload:
// complex128 ran fastest with the small tile on every step, FP32 pairs with
// this per-step choice).
double small_tile_cost(int precision) { return precision == ND_PREC_FP64 ? 0.9 : 1.15; }
// FP32 pairs: launches whose largest block edge exceeds TC_MIN_DIM take the
// tensor cores by default (their 128 x 64 tiles pad smaller blocks too much),
// unless the digit planes of the launch exceed TC_MAX_SCRATCH bytes per
// energy (thin blocks with many columns, as in the phonon G^< products).
// Measured on the 512 x 128 workload, 128 energies, GEMM time per size class
// (FP32 pipe -> tensor cores): edges in (96, 192]: 138.0 -> 170.5 ms,
// > 192: 139.9 -> 99.0 ms.
constexpr int TC_MIN_DIM = 192;
constexpr int64_t TC_MAX_SCRATCH = int64_t(512) << 20;
// ... and unless the planes of all energies of the handle exceed
// TC_TOTAL_SCRATCH (the 512-energy calls of the nanotube would otherwise ask
// for a few hundred GB).
constexpr int64_t TC_TOTAL_SCRATCH = int64_t(64) << 30;
bool tc_scratch_fits(int64_t per_energy, int max_ne) {
  return per_energy <= TC_MAX_SCRATCH && per_energy * int64_t(max_ne) <= TC_TOTAL_SCRATCH;
}
// Largest block edge of a GEMM launch that runs one CTA per block
// (k_gemm_direct).  Measured per size class on the 512 x 128 workload, FP32
// pairs, 128 energies (tiled 16 x 16 -> direct): edges <= 24: 78 -> 31 ms,
// <= 48: 47.5 -> 30.6 ms, <= 96: 74.9 -> 63.4 ms, <= 192: 138 -> 323 ms.
constexpr int DIRECT_MAX = 96;
// Above DIRECT_SMALL the direct kernel needs many blocks per launch (it runs
// one CTA per block and energy, each doing much sequential work): measured on
// the 256 x 64 superlattice, 128 energies, edges in (48, 96] with 16 blocks
// per launch: direct 32.4 ms, tiled 24.7 ms per call; on the 512 x 128 one,
// 163 blocks per launch: direct 63.4 ms, tiled 74.9 ms.  With this rule:
// 23.3 and 59.0 ms.
constexpr int DIRECT_SMALL = 48;
constexpr int64_t DIRECT_MIN_CTAS = 8192;

struct TcTables {
  std::vector<TcDesc> desc;
  std::vector<TcSplit> split;
  int64_t bytes = 0;  // largest per-energy scratch of a step
};

// Kernel of a GEMM step chosen by the tuner (nd_autotune): -1 = the default
// rules below, else a TileRange kind (0 large tile, 1 small tile, 2 tensor
// cores, 3 one CTA per block, 4 extra-large tile).
using Choice = std::vector<int8_t>;

// Per-energy digit scratch of a step on the tensor cores (bytes).
int64_t tc_step_scratch(const Step& s, const std::vector<GemmDesc>& gd) {
  int64_t off = 0;
  for (int k = s.begin; k < s.begin + s.count; ++k) {
    TcDesc t{};
    off = gemm_tc_scratch(gd[k], t, off);
  }
  return off;
}

// Tile edges (rows, columns) of the three ALU tile variants: large, small, extra large.
struct TileShapes {
  int m[3], n[3];
};

void build_tiles(const std::vector<Step>& sched, const std::vector<GemmDesc>& gd, const TileShapes& ts, int flags,
                 double small_cost, bool tc_ok, int max_ne, TcTables& tct, std::vector<TileRef>& tiles,
                 std::vector<TileRange>& ranges, const Choice* forced = nullptr) {
  const int tile_l = ts.m[0], tile_s = ts.m[1];
  ranges.assign(sched.size(), TileRange{0, 0, 0, 0, 0, 0});
  auto work = [&](const Step& s, int tile) {
    double w = 0.0;
    for (int k = s.begin; k < s.begin + s.count; ++k) {
      const GemmDesc& g = gd[k];
      w += double((g.m + tile - 1) / tile) * ((g.n + tile - 1) / tile) * tile * tile * std::max(1, g.k);
    }
    return w;
  };
  for (size_t si = 0; si < sched.size(); ++si) {
    const Step& s = sched[si];
    if (s.kind != ST_GEMM) continue;
    bool small = small_cost * work(s, tile_s) < work(s, tile_l);
    if (flags & ND_FACT_TILE_LARGE) small = false;
    if (flags & ND_FACT_TILE_SMALL) small = true;
    bool tc = false;
    if (tc_ok && !(flags & ND_FACT_GEMM_ALU)) {
      tc = !(flags & (ND_FACT_TILE_LARGE | ND_FACT_TILE_SMALL | ND_FACT_TILE_XL)) && s.max_dim > TC_MIN_DIM;
      if (tc) {
        int64_t off = 0;
        for (int k = s.begin; k < s.begin + s.count; ++k) {
          TcDesc t{};
          off = gemm_tc_scratch(gd[k], t, off);
        }
        tc = tc_scratch_fits(off, max_ne);
      }
      if (flags & ND_FACT_GEMM_TC) tc = true;
    }
    // launches whose blocks all have edges <= DIRECT_MAX take one CTA per block
    int dim = 0;
    for (int k = s.begin; k < s.begin + s.count; ++k) dim = std::max(dim, std::max(gd[k].m, std::max(gd[k].n, gd[k].k)));
    bool direct = !tc && !(flags & (ND_FACT_TILE_LARGE | ND_FACT_TILE_SMALL | ND_FACT_TILE_XL)) && dim <= DIRECT_MAX &&
                  (dim <= DIRECT_SMALL || int64_t(s.count) * max_ne >= DIRECT_MIN_CTAS);
    int variant = small ? 1 : 0;  // ALU tile variant
    if (flags & ND_FACT_TILE_XL) {
      variant = 2;
      direct = false;
    }
    if (forced && (*forced)[si] >= 0) {  // the tuner's measured choice
      const int c = (*forced)[si];
      tc = c == 2;
      direct = c == 3;
      variant = c == 1 ? 1 : c == 4 ? 2 : 0;
    }
    const int tmr = ts.m[variant], tnc = ts.n[variant];
    int b = int(tiles.size());
    if (tc) {
      const int sb = int(tct.split.size());
      int64_t off = 0;
      for (int k = s.begin; k < s.begin + s.count; ++k) {
        TcDesc t{};
        t.desc = k;
        off = gemm_tc_scratch(gd[k], t, off);
        const int ti = int(tct.desc.size());
        tct.desc.push_back(t);
        for (int r0 = 0; r0 < t.rba * TC_M; r0 += 32) tct.split.push_back(TcSplit{ti, 0, r0, 0});
        for (int r0 = 0; r0 < t.rbb * TC_N; r0 += 32) tct.split.push_back(TcSplit{ti, 1, r0, 0});
        for (int i = 0; i < t.rba; ++i)
          for (int j = 0; j < t.rbb; ++j) tiles.push_back(TileRef{ti, i, j, 0});
      }
      tct.bytes = std::max(tct.bytes, off);
      ranges[si] = TileRange{b, int(tiles.size()) - b, 2, sb, int(tct.split.size()) - sb, s.max_dim};
      continue;
    }
    for (int k = s.begin; k < s.begin + s.count; ++k) {
      const GemmDesc& g = gd[k];
      if (direct) {
        tiles.push_back(TileRef{k, 0, 0, 0});
        continue;
      }
      const int tm = (g.m + tmr - 1) / tmr, tn = (g.n + tnc - 1) / tnc;
      for (int i = 0; i < tm; ++i)
        for (int j = 0; j < tn; ++j) tiles.push_back(TileRef{k, i, j, 0});
    }
    ranges[si] = TileRange{b, int(tiles.size()) - b, direct ? 3 : variant == 1 ? 1 : variant == 2 ? 4 : 0, 0, 0, dim};
  }
}

// Copy a per-energy input (host or device memory) into the handle's buffer on
// the stream; the handle keeps it for the certificate of the same call.
nd_status stage_in(const double* src, double* staging, size_t bytes, cudaStream_t s, const double** out) {
  if (!src) {
    *out = nullptr;
    return ND_OK;
  }
  ND_CUDA(cudaMemcpyAsync(staging, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s));
  *out = staging;
  return ND_OK;
}

// Runs `body` on the caller's stream s, or, with ND_FACT_GRAPH (and the
// profiler off), replays the graph recorded for `key`, recording it first by
// running body on the private capture stream under stream capture.  Every
// pointer and scalar the launches of body take must be fixed by the key.
template <typename F>
nd_status graph_run(nd_fact* f, const uint64_t key[2], cudaStream_t s, F&& body) {
  if (!(f->flags & ND_FACT_GRAPH) || f->prof.on) return body(s);
  for (auto& g : f->graphs)
    if (g.key[0] == key[0] && g.key[1] == key[1]) {
      ND_CUDA(cudaGraphLaunch(g.exec, s));
      return ND_OK;
    }
  if (f->graphs.size() >= 16) f->clear_graphs();
  cudaStream_t c = f->cap_stream;
  ND_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeRelaxed));
  const nd_status st = body(c);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(c, &g);
  if (st != ND_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ee != cudaSuccess) return fail(ND_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(ND_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  f->graphs.push_back(nd_fact::GraphEntry{{key[0], key[1]}, exec});
  ND_CUDA(cudaGraphLaunch(exec, s));
  return ND_OK;
}

template <typename T>
nd_status run_schedule(nd_fact* f, const std::vector<Step>& sched, const std::vector<TileRange>& tr,
                       const Work& w, const double* ph_l, const double* ph_g, cudaStream_t s, int variant = 0,
                       const std::vector<double>* step_flops = nullptr) {
  const nd_plan* p = f->plan;
  const AncTables at{f->d_site_ids, f->d_unk_q, f->d_unk_r, f->d_anc_q,       f->d_anc_r,
                     f->d_cl_n,     f->d_cl_A,  f->d_cl_ldG, f->d_cl_offG, f->d_cl_offGX[variant]};
  const DelayTabs& dt = f->dt;
  for (size_t si = 0; si < sched.size(); ++si) {
    const Step& st = sched[si];
    Profiler::Rec rec{};
    if (f->prof.on) {
      // GEMM launches are recorded per kernel: "gemm" (large tile), "gemm_tc"
      // (tensor cores, kind 12), "gemm_small", "gemm_direct", "gemm_xl" (13-15)
      rec.kind = st.kind;
      if (st.kind == ST_GEMM) {
        const int k = tr[si].kind;
        rec.kind = k == 2 ? PROF_GEMM_TC : k == 1 ? PROF_GEMM_TC + 1 : k == 3 ? PROF_GEMM_TC + 2 : k == 4 ? PROF_GEMM_TC + 3 : ST_GEMM;
      }
      rec.a = f->prof.get();
      rec.b = f->prof.get();
      rec.flops = step_flops ? (*step_flops)[si] * w.n_e : 0.0;
      rec.bytes = 0.0;
      rec.count = st.count;
      rec.max_dim = st.max_dim;
      rec.n_e = w.n_e;
      rec.tr = &tr;
      rec.si = int(si);
      cudaEventRecord(rec.a, s);
    }
    switch (st.kind) {
      case ST_INVERSE:
        Kern<T>::inverse(w, f->d_inv + st.begin, st.count, st.max_dim, f->root_scratch, f->root_stride, f->d_status,
                         s);
        break;
      case ST_GEMM:
        if (tr[si].kind == 2)
          launch_gemm_tc(w, f->d_gemm, f->d_tcd, f->d_tcsplit + tr[si].sfirst, tr[si].scount,
                         f->d_tiles + tr[si].first, tr[si].count, f->tc_scratch, f->tc_stride, f->d_tc_timeout,
                         f->tc_wait_polls, s);
        else if (tr[si].kind == 3)
          Kern<T>::gemm_direct(w, f->d_gemm, f->d_tiles + tr[si].first, tr[si].count, s);
        else
          Kern<T>::gemm(w, f->d_gemm, f->d_tiles + tr[si].first, tr[si].count,
                        tr[si].kind == 1 ? 1 : tr[si].kind == 4 ? 2 : 0, s);
        break;
      case ST_SCATTER:
        Kern<T>::scatter(w, f->d_scat + st.begin, st.count, f->d_maps, s);
        break;
      case ST_GATHER_SYM:
      case ST_GATHER_SKEW:
        Kern<T>::gather(w, f->d_gath + st.begin, st.count, f->d_maps, st.kind == ST_GATHER_SKEW, dt, s);
        break;
      case ST_ZERO:
        Kern<T>::zero(w, f->d_zero + st.begin, st.count, s);
        break;
      case ST_NPH:
        Kern<T>::nph(w, f->d_nph + st.begin, st.count, f->d_sites, ph_l, ph_g, p->n, dt, s);
        break;
      case ST_GATHER_ANC:
        Kern<T>::gather_anc(w, f->d_anc + st.begin, st.count, at, dt, s);
        break;
      case ST_SCATTER_ROWS:
        Kern<T>::scatter_rows(w, f->d_rows + st.begin, st.count, f->d_maps, dt, s);
        break;
      case ST_COLGATHER:
        Kern<T>::colgather(w, f->d_colg + st.begin, st.count, f->d_cmaps, at, dt, s);
        break;
      case ST_DELAY:
        Kern<T>::delay(w, f->d_delay + st.begin, st.count, st.max_dim, dt, s);
        break;
      case ST_LOC:
        launch_loc(f->d_loc + st.begin, st.count, w.n_e, dt, s);
        break;
      case ST_ROWS_ADD:
      case ST_ROWS_GATHER:
        Kern<T>::rows(w, f->d_rows_adj + st.begin, st.count, f->d_maps, p->adj_cols, st.kind == ST_ROWS_GATHER, dt, s);
        break;
    }
    if (f->prof.on) {
      cudaEventRecord(rec.b, s);
      f->prof.recs.push_back(rec);
    }
  }
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

// Algorithmic flops per energy of every step (8 per complex multiply-add for
// GEMMs, n^3 complex multiply-adds per inverse); 0 for data movement steps.
std::vector<double> step_flops(const nd_plan* p, const std::vector<Step>& sched,
                               const std::vector<GemmDesc>* gemms = nullptr) {
  const std::vector<GemmDesc>& gd = gemms ? *gemms : p->gemm_desc;
  std::vector<double> out(sched.size(), 0.0);
  for (size_t si = 0; si < sched.size(); ++si) {
    const Step& st = sched[si];
    double f = 0.0;
    if (st.kind == ST_GEMM)
      for (int k = st.begin; k < st.begin + st.count; ++k) {
        const GemmDesc& g = gd[k];
        f += 8.0 * double(g.m) * g.n * g.k;
      }
    if (st.kind == ST_INVERSE)
      for (int k = st.begin; k < st.begin + st.count; ++k) {
        const double n = p->inv_desc[k].n;
        f += 8.0 * n * n * n;
      }
    if (st.kind == ST_DELAY)  // complex64 inverse of the front's interior block and k rank-one updates
      for (int k = st.begin; k < st.begin + st.count; ++k) {
        const double n = p->delay_desc[k].nf;
        f += 8.0 * n * n * (n + p->delay_desc[k].k);
      }
    out[si] = f;
  }
  return out;
}

// Schedules of the adjoint solves (nd_density_gradient), appended to the
// GEMM table: per level, upward RB += Psi^T XI then the rows of RB into the
// parent (one launch per child slot); downward the boundary rows from the
// parent, XS = A_ii^{-1} XI, XS += Psi XB.  Offsets are per-energy elements,
// `base` the start of the adjoint blocks in the workspace.
void build_adjoint(const nd_plan* p, int64_t base, std::vector<GemmDesc>& gemms, std::vector<RowsDesc>& rows,
                   std::vector<Step>& fwd, std::vector<Step>& bwd, std::vector<AdjDesc>& adesc,
                   std::vector<int64_t>& ones) {
  const auto& cl = p->cl;
  const int nc = int(cl.size());
  const int M = p->adj_cols;
  std::vector<int32_t> site_begin(nc), map_begin(nc);
  int32_t sb = 0, mb = 0;
  for (int i = 0; i < nc; ++i) {
    site_begin[i] = sb;
    map_begin[i] = mb;
    sb += cl[i].nf();
    mb += int32_t(cl[i].map.size());
  }
  std::vector<std::vector<int>> lev(p->n_levels + 1);
  int max_slot = 0;
  for (int i = 0; i < nc; ++i) {
    lev[cl[i].level].push_back(i);
    max_slot = std::max(max_slot, cl[i].slot);
  }
  auto gemm = [&](int64_t C, int ldc, int64_t D, int ldd, int64_t A, int lda, int opA, int64_t B, int ldb, int m,
                  int n, int k, double beta) {
    GemmDesc g{};
    g.offA = A; g.offB = B; g.offC = C; g.offD = D;
    g.m = m; g.n = n; g.k = k;
    g.lda = lda; g.ldb = ldb; g.ldc = ldc; g.ldd = ldd;
    g.opA = opA; g.opB = OP_N;
    g.alpha = 1.0; g.beta = beta;
    gemms.push_back(g);
  };
  auto step = [&](std::vector<Step>& S, int kind, int begin, int end, int dim) {
    if (end > begin) S.push_back(Step{kind, begin, end - begin, dim});
  };
  for (int l = 1; l <= p->n_levels; ++l) {
    int b0 = int(gemms.size()), dim = 0;
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0 || c.n == 0) continue;
      gemm(base + c.adj_RB, M, base + c.adj_RB, M, c.off_Psi, c.b, OP_T, base + c.adj_XI, M, c.b, M, c.n, 1.0);
      dim = std::max(dim, std::max(c.n, std::max(c.b, M)));
    }
    step(fwd, ST_GEMM, b0, int(gemms.size()), dim);
    for (int sl = 0; sl <= max_slot; ++sl) {
      int r0 = int(rows.size());
      dim = 0;
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0 || c.slot != sl) continue;
        const Cluster& P = cl[c.parent];
        rows.push_back(RowsDesc{base + c.adj_RB, base + P.adj_XI, base + P.adj_RB, c.b, P.n, P.k,
                                site_begin[c.parent], map_begin[i]});
        dim = std::max(dim, c.b);
      }
      step(fwd, ST_ROWS_ADD, r0, int(rows.size()), dim);
    }
  }
  for (int l = p->n_levels; l >= 1; --l) {
    int r0 = int(rows.size()), dim = 0;
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const Cluster& P = cl[c.parent];
      rows.push_back(RowsDesc{base + c.adj_XB, base + P.adj_XS, base + P.adj_XB, c.b, P.n, P.k, site_begin[c.parent],
                              map_begin[i]});
      dim = std::max(dim, c.b);
    }
    step(bwd, ST_ROWS_GATHER, r0, int(rows.size()), dim);
    int b0 = int(gemms.size());
    dim = 0;
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.n == 0) continue;
      gemm(base + c.adj_XS, M, base + c.adj_XS, M, c.off_F, c.n + c.b, OP_N, base + c.adj_XI, M, c.n, M, c.n, 0.0);
      dim = std::max(dim, std::max(c.n, M));
    }
    step(bwd, ST_GEMM, b0, int(gemms.size()), dim);
    b0 = int(gemms.size());
    dim = 0;
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0 || c.n == 0) continue;
      gemm(base + c.adj_XS, M, base + c.adj_XS, M, c.off_Psi, c.b, OP_N, base + c.adj_XB, M, c.n, M, c.b, 1.0);
      dim = std::max(dim, std::max(c.b, std::max(c.n, M)));
    }
    step(bwd, ST_GEMM, b0, int(gemms.size()), dim);
  }
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = cl[i];
    adesc.push_back(AdjDesc{base + c.adj_XI, base + c.adj_RB, base + c.adj_XS, base + c.adj_U, c.n, c.b,
                            site_begin[i], 0});
  }
  for (int ct = 0; ct < p->n_contacts; ++ct) {
    const Cluster& c = cl[p->contact_cluster[ct]];
    const int m = p->contact_ptr[ct + 1] - p->contact_ptr[ct];
    for (int a = 0; a < m; ++a)
      ones.push_back(base + c.adj_XI + int64_t(p->contact_row[ct] + a) * M + p->contact_ptr[ct] + a);
  }
}

}  // namespace

// Schedules whose GEMM steps carry a tile list, in a fixed order (the tuner's
// choices are indexed by it): factor, G^r, G^< without / with phonons, and the
// adjoint solves.
constexpr int N_SCHED = 6;

void free_tracked(nd_fact* f, void* p) {
  if (!p) return;
  auto it = std::find(f->allocs.begin(), f->allocs.end(), p);
  if (it != f->allocs.end()) f->allocs.erase(it);
  cudaFree(p);
}

// Tile lists of every GEMM step (default rules, or the choices of
// nd_autotune), uploaded with the tensor-core tables; the digit scratch grows
// when the new choices need more.
nd_status build_all_tiles(nd_fact* f, const std::array<Choice, N_SCHED>* forced) {
  const nd_plan* p = f->plan;
  const int precision = f->precision, flags = f->flags, max_ne = f->max_ne;
  TileShapes tsh;
  for (int v = 0; v < 3; ++v) {
    tsh.m[v] = precision == ND_PREC_FP64    ? Kern<double>::gemm_tile(v)
               : precision == ND_PREC_MIXED ? Kern<float>::gemm_tile(v)
                                            : Kern<DF>::gemm_tile(v);
    tsh.n[v] = precision == ND_PREC_FP64    ? Kern<double>::gemm_tile_n(v)
               : precision == ND_PREC_MIXED ? Kern<float>::gemm_tile_n(v)
                                            : Kern<DF>::gemm_tile_n(v);
  }
  std::vector<TileRef> tiles;
  const double sc = small_tile_cost(precision);
  const bool tc_ok = precision == ND_PREC_FP32X2;
  const bool ph = (flags & ND_FACT_PHONON) != 0;  // the phonon G^< schedule runs only on a phonon workspace
  TcTables tct;
  auto fc = [&](int q) { return forced ? &(*forced)[q] : nullptr; };
  build_tiles(p->sched_factor, f->gemm_all, tsh, flags, sc, tc_ok, max_ne, tct, tiles, f->tr_factor, fc(0));
  build_tiles(p->sched_green, f->gemm_all, tsh, flags, sc, tc_ok, max_ne, tct, tiles, f->tr_green, fc(1));
  build_tiles(p->sched_lesser[0], f->gemm_all, tsh, flags, sc, tc_ok, max_ne, tct, tiles, f->tr_lesser[0], fc(2));
  build_tiles(p->sched_lesser[1], f->gemm_all, tsh, flags, sc, tc_ok && ph, max_ne, tct, tiles, f->tr_lesser[1],
              fc(3));
  if (f->adj) {
    build_tiles(f->sched_adj_fwd, f->gemm_all, tsh, flags, sc, tc_ok, max_ne, tct, tiles, f->tr_adj_fwd, fc(4));
    build_tiles(f->sched_adj_bwd, f->gemm_all, tsh, flags, sc, tc_ok, max_ne, tct, tiles, f->tr_adj_bwd, fc(5));
  }
  free_tracked(f, f->d_tiles);
  free_tracked(f, f->d_tcd);
  free_tracked(f, f->d_tcsplit);
  f->d_tiles = nullptr;
  f->d_tcd = nullptr;
  f->d_tcsplit = nullptr;
  nd_status st;
  if ((st = dupload(f, tiles, &f->d_tiles)) != ND_OK) return st;
  if (!tct.desc.empty()) {
    if ((st = dupload(f, tct.desc, &f->d_tcd)) != ND_OK) return st;
    if ((st = dupload(f, tct.split, &f->d_tcsplit)) != ND_OK) return st;
    if (tct.bytes > f->tc_stride || !f->tc_scratch) {
      free_tracked(f, f->tc_scratch);
      f->tc_scratch = nullptr;
      f->tc_stride = tct.bytes;
      if ((st = dalloc(f, (void**)&f->tc_scratch, size_t(tct.bytes) * size_t(max_ne))) != ND_OK) return st;
    }
  }
  f->clear_graphs();
  return ND_OK;
}

extern "C" nd_status nd_fact_create(const nd_plan* p, int32_t max_ne, int32_t precision, int32_t flags,
                                    nd_fact** out) {
  if (!p || !out || max_ne <= 0) return fail(ND_ERR_INVALID_ARG, "nd_fact_create: bad argument");
  if (precision != ND_PREC_FP64 && precision != ND_PREC_MIXED && precision != ND_PREC_FP32X2)
    return fail(ND_ERR_INVALID_ARG, "nd_fact_create: unknown precision");
  if (p->max_n > 8192) return fail(ND_ERR_UNSUPPORTED, "nd_fact_create: cluster larger than 8192 sites");
  if (p->max_b > 32768) return fail(ND_ERR_UNSUPPORTED, "nd_fact_create: cluster boundary larger than 32768 sites");
  for (const auto& c : p->cl)
    if (c.contacts.size() > 2) return fail(ND_ERR_UNSUPPORTED, "nd_fact_create: more than two contacts in one cluster");
  *out = nullptr;
  auto f = new nd_fact();
  f->plan = p;
  f->precision = precision;
  f->max_ne = max_ne;
  f->esize = precision == ND_PREC_MIXED ? 8 : 16;
  f->flags = flags;
  f->se = p->arena_elems + ((flags & ND_FACT_PHONON) ? std::max(p->ext_elems[0], p->ext_elems[1]) : p->ext_elems[0]);
  if (flags & ND_FACT_ADJOINT) {  // the adjoint blocks follow the rest of each energy's workspace
    f->adj = true;
    f->adj_base = f->se;
    f->se += p->adj_elems;
  }
  nd_status st;
#define TRY(x)          \
  do {                  \
    st = (x);           \
    if (st != ND_OK) {  \
      delete f;         \
      return st;        \
    }                   \
  } while (0)
  TRY(dalloc(f, &f->arena, size_t(f->se) * f->esize * max_ne));
  TRY(dalloc(f, &f->aux, size_t(std::max<int64_t>(1, 2 * p->sigma_elems)) * f->esize * max_ne));
  if (precision != ND_PREC_FP64) {  // one complex128 region per root block and energy
    f->root_stride = p->root_scratch_elems;
    TRY(dalloc(f, (void**)&f->root_scratch, size_t(p->root_scratch_elems) * 16 * max_ne));
  }
  TRY(dalloc(f, (void**)&f->d_status, sizeof(int)));
  cudaMemset(f->d_status, 0, sizeof(int));
  TRY(dalloc(f, (void**)&f->d_inerr, 2 * sizeof(int)));
  cudaMemset(f->d_inerr, 0, 2 * sizeof(int));
  TRY(dupload(f, p->csr_T, &f->d_csrT));
  {
    std::vector<int32_t> cm(p->n_contacts);
    for (int c = 0; c < p->n_contacts; ++c) cm[c] = p->contact_ptr[c + 1] - p->contact_ptr[c];
    TRY(dupload(f, cm, &f->d_cm));
    TRY(dupload(f, p->contact_soff, &f->d_csoff));
  }
  TRY(dupload(f, p->sites, &f->d_sites));
  TRY(dupload(f, p->maps, &f->d_maps));
  TRY(dupload(f, p->ent_dst, &f->d_ent_dst));
  TRY(dupload(f, p->ent_src, &f->d_ent_src));
  TRY(dupload(f, p->asm_desc, &f->d_asm));
  TRY(dupload(f, p->inv_desc, &f->d_inv));
  std::vector<GemmDesc> gemm_all = p->gemm_desc;
  if (f->adj) {
    std::vector<RowsDesc> rows;
    std::vector<AdjDesc> adesc;
    std::vector<int64_t> ones;
    build_adjoint(p, f->adj_base, gemm_all, rows, f->sched_adj_fwd, f->sched_adj_bwd, adesc, ones);
    TRY(dupload(f, rows, &f->d_rows_adj));
    TRY(dupload(f, adesc, &f->d_adj_desc));
    TRY(dupload(f, ones, &f->d_ones));
    f->n_adj_desc = int(adesc.size());
    f->n_ones = int(ones.size());
    TRY(dalloc(f, (void**)&f->d_cvec, size_t(std::max(1, p->n)) * sizeof(double)));
    f->step_flops_adj_fwd = step_flops(p, f->sched_adj_fwd, &gemm_all);
    f->step_flops_adj_bwd = step_flops(p, f->sched_adj_bwd, &gemm_all);
  }
  TRY(dupload(f, gemm_all, &f->d_gemm));
  f->gemm_all = gemm_all;
  TRY(dupload(f, p->scat_desc, &f->d_scat));
  TRY(dupload(f, p->gath_desc, &f->d_gath));
  TRY(dupload(f, p->diag_g, &f->d_diag_g));
  TRY(dupload(f, p->diag_p[0], &f->d_diag_p[0]));
  TRY(dupload(f, p->diag_p[1], &f->d_diag_p[1]));
  TRY(dupload(f, p->nph_desc, &f->d_nph));
  TRY(dupload(f, p->zero_desc, &f->d_zero));
  TRY(dupload(f, p->anc_desc, &f->d_anc));
  TRY(dupload(f, p->rows_desc, &f->d_rows));
  TRY(dupload(f, p->colg_desc, &f->d_colg));
  TRY(dupload(f, p->delay_desc, &f->d_delay));
  TRY(dupload(f, p->loc_desc, &f->d_loc));
  TRY(dupload(f, p->unk_q, &f->d_unk_q));
  TRY(dupload(f, p->unk_r, &f->d_unk_r));
  TRY(dupload(f, p->anc_q, &f->d_anc_q));
  TRY(dupload(f, p->anc_r, &f->d_anc_r));
  if (p->n_virtual > 0) {
    const size_t tb = size_t(p->n_unk) * max_ne * sizeof(int32_t);
    f->dt.n_unk = p->n_unk;
    TRY(dalloc(f, (void**)&f->dt.iperm, tb));
    TRY(dalloc(f, (void**)&f->dt.rsite, tb));
    TRY(dalloc(f, (void**)&f->dt.locq, tb));
    TRY(dalloc(f, (void**)&f->dt.locr, tb));
  }
  TRY(dupload(f, p->site_ids, &f->d_site_ids));
  TRY(dupload(f, p->cmaps, &f->d_cmaps));
  TRY(dupload(f, p->owner, &f->d_owner));
  TRY(dupload(f, p->pos, &f->d_pos));
  TRY(dupload(f, p->cl_n, &f->d_cl_n));
  TRY(dupload(f, p->cl_A, &f->d_cl_A));
  TRY(dupload(f, p->cl_ldG, &f->d_cl_ldG));
  TRY(dupload(f, p->cl_offG, &f->d_cl_offG));
  TRY(dupload(f, p->cl_offGX[0], &f->d_cl_offGX[0]));
  TRY(dupload(f, p->cl_offGX[1], &f->d_cl_offGX[1]));
  TRY(dupload(f, p->cert_ptr, &f->d_cert_ptr));
  TRY(dupload(f, p->cert_nb, &f->d_cert_nb));
  TRY(dupload(f, p->cert_coef, &f->d_cert_coef));
  TRY(dupload(f, p->cert_slot, &f->d_cert_slot));
  TRY(dupload(f, p->cert_bslot, &f->d_cert_bslot));
  TRY(dupload(f, p->cert_bidx, &f->d_cert_bidx));
  TRY(dupload(f, p->cert_cl, &f->d_cert_cl));
  TRY(dalloc(f, (void**)&f->d_cert, size_t(max_ne) * 8 * sizeof(double)));
  TRY(dalloc(f, (void**)&f->d_current, size_t(max_ne) * 2 * sizeof(double)));
  TRY(dalloc(f, (void**)&f->d_w, size_t(max_ne) * sizeof(double)));
  TRY(dalloc(f, (void**)&f->d_dens, size_t(std::max(1, p->n)) * sizeof(double)));
  TRY(dupload(f, p->psi_desc, &f->d_psi));
  f->step_flops_factor = step_flops(p, p->sched_factor);
  f->step_flops_green = step_flops(p, p->sched_green);
  f->step_flops_lesser[0] = step_flops(p, p->sched_lesser[0]);
  f->step_flops_lesser[1] = step_flops(p, p->sched_lesser[1]);
  TRY(build_all_tiles(f, nullptr));
  TRY(dalloc(f, (void**)&f->d_tc_timeout, sizeof(int)));
  cudaMemset(f->d_tc_timeout, 0, sizeof(int));
  const size_t ne = size_t(max_ne), n = size_t(p->n), se = size_t(p->sigma_elems);
  TRY(dalloc(f, (void**)&f->st_H, size_t(std::max(1, p->nnz)) * 8));
  TRY(dalloc(f, (void**)&f->st_sr, std::max<size_t>(1, ne * se) * 16));
  TRY(dalloc(f, (void**)&f->st_ph, ne * n * 16));
  TRY(dalloc(f, (void**)&f->st_E, ne * 8));
  TRY(dalloc(f, (void**)&f->st_sl, std::max<size_t>(1, ne * se) * 16));
  TRY(dalloc(f, (void**)&f->st_sg, std::max<size_t>(1, ne * se) * 16));
  TRY(dalloc(f, (void**)&f->st_pl, ne * n * 16));
  TRY(dalloc(f, (void**)&f->st_pg, ne * n * 16));
  for (int k = 0; k < 3; ++k) TRY(dalloc(f, (void**)&f->st_out[k], ne * n * 16));
#undef TRY
  if (flags & ND_FACT_GRAPH) {
    if (cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete f;
      return fail(ND_ERR_CUDA, "nd_fact_create: cannot create the capture stream");
    }
  }
  prepare_kernels();  // function attributes are set here, never during a capture
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete f;
    return fail(ND_ERR_CUDA, std::string("nd_fact_create: ") + cudaGetErrorString(e));
  }
  *out = f;
  return ND_OK;
}

extern "C" void nd_fact_destroy(nd_fact* f) { delete f; }

template <typename T>
static nd_status factor_t(nd_fact* f, const Work& w, const double* H, const double* E, double eta, const double* sr,
                          const double* ph, int nc, cudaStream_t s) {
  const nd_plan* p = f->plan;
  Kern<T>::assemble(w, f->d_asm, nc, f->d_ent_dst, f->d_ent_src, f->d_sites, H, E, eta, sr, p->sigma_elems, ph, p->n,
                    f->dt, s);
  return run_schedule<T>(f, p->sched_factor, f->tr_factor, w, nullptr, nullptr, s, 0, &f->step_flops_factor);
}

extern "C" nd_status nd_factor(nd_fact* f, const double* H_values, const double* sigma_r, const double* sigma_ph_r,
                               const double* energies, int32_t n_e, double eta, void* stream) {
  if (!f || !H_values || !energies) return fail(ND_ERR_INVALID_ARG, "nd_factor: NULL argument");
  if (n_e <= 0 || n_e > f->max_ne) return fail(ND_ERR_INVALID_ARG, "nd_factor: n_e outside 1..max_ne");
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ND_ERR_INVALID_ARG, "nd_factor: eta must be positive and finite");
  const nd_plan* p = f->plan;
  if (p->n_contacts > 0 && !sigma_r) return fail(ND_ERR_INVALID_ARG, "nd_factor: sigma_r is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const double *H, *sr, *ph, *E;
  nd_status st;
  // complex symmetry of A (paper Sec. 3.1): host inputs are checked here, device inputs on the stream below
  const bool H_dev = is_device_ptr(H_values), sr_dev = p->n_contacts > 0 && is_device_ptr(sigma_r);
  if ((st = host_check_factor(p, H_dev ? nullptr : H_values, (p->n_contacts > 0 && !sr_dev) ? sigma_r : nullptr,
                              n_e)) != ND_OK)
    return fail(st, std::string("nd_factor: ") + nd_last_error());
  if ((st = stage_in(H_values, f->st_H, size_t(p->nnz) * 8, s, &H)) != ND_OK) return st;
  if ((st = stage_in(sigma_r, f->st_sr, size_t(n_e) * p->sigma_elems * 16, s, &sr)) != ND_OK) return st;
  if ((st = stage_in(sigma_ph_r, f->st_ph, size_t(n_e) * p->n * 16, s, &ph)) != ND_OK) return st;
  if ((st = stage_in(energies, f->st_E, size_t(n_e) * 8, s, &E)) != ND_OK) return st;
  f->n_e = n_e;
  f->eta = eta;
  f->cur_H = H;
  f->cur_sr = sr;
  f->cur_ph = ph;
  f->cur_E = E;
  f->have_lesser = false;
  f->have_green = false;
  f->adj_u_valid = false;
  f->last_gl = nullptr;
  ND_CUDA(cudaMemsetAsync(f->d_status, 0, sizeof(int), s));
  ND_CUDA(cudaMemsetAsync(f->d_tc_timeout, 0, sizeof(int), s));
  ND_CUDA(cudaMemsetAsync(f->d_inerr, 0, 2 * sizeof(int), s));
  if (H_dev) launch_check_H(H, f->d_csrT, p->nnz, f->d_inerr, s);
  if (sr_dev) launch_check_blocks(sr, p->sigma_elems, f->d_csoff, f->d_cm, p->n_contacts, n_e, false, f->d_inerr, s);
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, n_e};
  const int nc = int(p->cl.size());
  uint64_t eta_bits;
  std::memcpy(&eta_bits, &eta, 8);
  const uint64_t key[2] = {(uint64_t(n_e) << 8) | (sr ? 2u : 0u) | (ph ? 4u : 0u), eta_bits};
  return graph_run(f, key, s, [&](cudaStream_t q) {
    if (f->precision == ND_PREC_FP64) return factor_t<double>(f, w, H, E, eta, sr, ph, nc, q);
    if (f->precision == ND_PREC_MIXED) return factor_t<float>(f, w, H, E, eta, sr, ph, nc, q);
    return factor_t<DF>(f, w, H, E, eta, sr, ph, nc, q);
  });
}

template <typename T>
static nd_status diag_green_t(nd_fact* f, const double* sl, const double* sg, const double* pl, const double* pg,
                              double* outs[3], cudaStream_t s) {
  const nd_plan* p = f->plan;
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, f->n_e};
  const int nc = int(p->cl.size());
  nd_status st = run_schedule<T>(f, p->sched_green, f->tr_green, w, nullptr, nullptr, s, 0, &f->step_flops_green);
  if (st != ND_OK) return st;
  if (outs[0]) Kern<T>::diag_out(w, f->d_diag_g, nc, f->d_sites, outs[0], p->n, f->dt, s);
  if (outs[1] || outs[2]) {
    Kern<T>::convert_aux(w, sl, sg, p->sigma_elems, s);
    const int v = (pl || pg) ? 1 : 0;
    st = run_schedule<T>(f, p->sched_lesser[v], f->tr_lesser[v], w, pl, pg, s, v, &f->step_flops_lesser[v]);
    if (st != ND_OK) return st;
    if (outs[1]) Kern<T>::diag_out(w, f->d_diag_p[0], nc, f->d_sites, outs[1], p->n, f->dt, s);
    if (outs[2]) Kern<T>::diag_out(w, f->d_diag_p[1], nc, f->d_sites, outs[2], p->n, f->dt, s);
  }
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_diag_green(nd_fact* f, const double* sigma_lesser, const double* sigma_greater,
                                   const double* ph_lesser, const double* ph_greater, double* Gr, double* Gl,
                                   double* Gg, void* stream) {
  if (!f) return fail(ND_ERR_INVALID_ARG, "nd_diag_green: NULL handle");
  if (f->n_e <= 0) return fail(ND_ERR_INVALID_ARG, "nd_diag_green: call nd_factor first");
  if ((Gl || Gg) && f->plan->n_contacts > 0 && !sigma_lesser && !sigma_greater && !ph_lesser && !ph_greater)
    return fail(ND_ERR_INVALID_ARG, "nd_diag_green: G^< / G^> requested without Sigma^< / Sigma^>");
  if ((ph_lesser == nullptr) != (ph_greater == nullptr))
    return fail(ND_ERR_INVALID_ARG, "nd_diag_green: pass both phonon Sigma^< and Sigma^> or neither");
  if (ph_lesser && !(f->flags & ND_FACT_PHONON))
    return fail(ND_ERR_INVALID_ARG, "nd_diag_green: phonon Sigma^< needs a workspace created with ND_FACT_PHONON");
  const nd_plan* p = f->plan;
  cudaStream_t s = (cudaStream_t)stream;
  const int n_e = f->n_e;
  const double *sl, *sg, *pl, *pg;
  nd_status st;
  // skew-Hermitian Sigma^< / Sigma^> (paper Sec. 3.1): host inputs here, device inputs on the stream below
  const bool has_c = p->n_contacts > 0;
  const bool dev_in[4] = {has_c && is_device_ptr(sigma_lesser), has_c && is_device_ptr(sigma_greater),
                          is_device_ptr(ph_lesser), is_device_ptr(ph_greater)};
  {
    const double* blocks[2] = {has_c && !dev_in[0] ? sigma_lesser : nullptr, has_c && !dev_in[1] ? sigma_greater : nullptr};
    const double* diags[2] = {dev_in[2] ? nullptr : ph_lesser, dev_in[3] ? nullptr : ph_greater};
    if ((st = host_check_lesser(p, blocks, diags, n_e)) != ND_OK)
      return fail(st, std::string("nd_diag_green: ") + nd_last_error());
  }
  ND_CUDA(cudaMemsetAsync(f->d_inerr + 1, 0, sizeof(int), s));
  if ((st = stage_in(sigma_lesser, f->st_sl, size_t(n_e) * p->sigma_elems * 16, s, &sl)) != ND_OK) return st;
  if ((st = stage_in(sigma_greater, f->st_sg, size_t(n_e) * p->sigma_elems * 16, s, &sg)) != ND_OK) return st;
  if ((st = stage_in(ph_lesser, f->st_pl, size_t(n_e) * p->n * 16, s, &pl)) != ND_OK) return st;
  if ((st = stage_in(ph_greater, f->st_pg, size_t(n_e) * p->n * 16, s, &pg)) != ND_OK) return st;
  if (dev_in[0]) launch_check_blocks(sl, p->sigma_elems, f->d_csoff, f->d_cm, p->n_contacts, n_e, true, f->d_inerr + 1, s);
  if (dev_in[1]) launch_check_blocks(sg, p->sigma_elems, f->d_csoff, f->d_cm, p->n_contacts, n_e, true, f->d_inerr + 1, s);
  if (dev_in[2]) launch_check_diag_skew(pl, int64_t(n_e) * p->n, f->d_inerr + 1, s);
  if (dev_in[3]) launch_check_diag_skew(pg, int64_t(n_e) * p->n, f->d_inerr + 1, s);
  double* user[3] = {Gr, Gl, Gg};
  double* dev[3];
  bool host[3], copy[3];
  const bool graph = (f->flags & ND_FACT_GRAPH) && !f->prof.on;
  for (int k = 0; k < 3; ++k) {
    host[k] = user[k] && !is_device_ptr(user[k]);
    copy[k] = user[k] && (host[k] || graph);  // with graphs the outputs always go through the staging buffers
    dev[k] = copy[k] ? f->st_out[k] : user[k];
  }
  const uint64_t key[2] = {(uint64_t(n_e) << 16) | 1u | (sl ? 2u : 0u) | (sg ? 4u : 0u) | (pl ? 8u : 0u) |
                               (pg ? 16u : 0u) | (Gr ? 32u : 0u) | (Gl ? 64u : 0u) | (Gg ? 128u : 0u),
                           0};
  st = graph_run(f, key, s, [&](cudaStream_t q) {
    return f->precision == ND_PREC_FP64    ? diag_green_t<double>(f, sl, sg, pl, pg, dev, q)
           : f->precision == ND_PREC_MIXED ? diag_green_t<float>(f, sl, sg, pl, pg, dev, q)
                                           : diag_green_t<DF>(f, sl, sg, pl, pg, dev, q);
  });
  if (st != ND_OK) return st;
  f->have_green = true;
  f->have_lesser = (Gl || Gg);
  f->last_gl = Gl ? dev[1] : nullptr;
  f->cur_sl = sl;
  f->cur_sg = sg;
  f->cur_pl = pl;
  for (int k = 0; k < 3; ++k)
    if (copy[k])
      ND_CUDA(cudaMemcpyAsync(user[k], dev[k], size_t(n_e) * p->n * 16,
                              host[k] ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  return ND_OK;
}

static CertArgs cert_args(nd_fact* f) {
  const nd_plan* p = f->plan;
  CertArgs a{};
  a.n = p->n;
  a.cptr = f->d_cert_ptr;
  a.nb = f->d_cert_nb;
  a.coef = f->d_cert_coef;
  a.slot = f->d_cert_slot;
  a.bslot = f->d_cert_bslot;
  a.bidx = f->d_cert_bidx;
  a.unk_q = f->d_unk_q;
  a.unk_r = f->d_unk_r;
  a.cl = f->d_cert_cl;
  a.H = f->cur_H;
  a.sr = f->cur_sr;
  a.sl = f->cur_sl;
  a.ph_r = f->cur_ph;
  a.ph_l = f->cur_pl;
  a.energies = f->cur_E;
  a.sstride = p->sigma_elems;
  a.eta = f->eta;
  a.lesser = f->have_lesser ? 1 : 0;
  a.cert = f->d_cert;
  a.psi = f->d_psi;
  a.n_psi = int(p->psi_desc.size());
  return a;
}

extern "C" nd_status nd_certificate(nd_fact* f, double* cert, void* stream) {
  if (!f || !cert) return fail(ND_ERR_INVALID_ARG, "nd_certificate: NULL argument");
  if (f->n_e <= 0 || !f->have_green)
    return fail(ND_ERR_INVALID_ARG, "nd_certificate: call nd_factor and nd_diag_green first");
  const nd_plan* p = f->plan;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = size_t(f->n_e) * 8 * sizeof(double);
  ND_CUDA(cudaMemsetAsync(f->d_cert, 0, bytes, s));
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, f->n_e};
  const CertArgs a = cert_args(f);
  if (f->precision == ND_PREC_FP64)
    Kern<double>::certificate(w, a, f->dt, s);
  else if (f->precision == ND_PREC_MIXED)
    Kern<float>::certificate(w, a, f->dt, s);
  else
    Kern<DF>::certificate(w, a, f->dt, s);
  ND_CUDA(cudaGetLastError());
  ND_CUDA(cudaMemcpyAsync(cert, f->d_cert, bytes, is_device_ptr(cert) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s));
  return ND_OK;
}

extern "C" nd_status nd_selected_entries(nd_fact* f, const int32_t* x, const int32_t* y, int32_t count, double* Gr,
                                         double* Gl, double* Gg, int32_t* n_missing, void* stream) {
  if (!f || !x || !y || !n_missing || count < 0) return fail(ND_ERR_INVALID_ARG, "nd_selected_entries: bad argument");
  if (f->n_e <= 0 || !f->have_green)
    return fail(ND_ERR_INVALID_ARG, "nd_selected_entries: call nd_factor and nd_diag_green first");
  if ((Gl || Gg) && !f->have_lesser)
    return fail(ND_ERR_INVALID_ARG, "nd_selected_entries: G^< / G^> need a preceding nd_diag_green that computed them");
  const void* dev[] = {x, y, n_missing};
  for (const void* q : dev)
    if (!is_device_ptr(q)) return fail(ND_ERR_INVALID_ARG, "nd_selected_entries: x, y, n_missing must be device arrays");
  const void* outs[] = {Gr, Gl, Gg};
  for (const void* q : outs)
    if (q && !is_device_ptr(q)) return fail(ND_ERR_INVALID_ARG, "nd_selected_entries: outputs must be device arrays");
  const nd_plan* p = f->plan;
  cudaStream_t s = (cudaStream_t)stream;
  ND_CUDA(cudaMemsetAsync(n_missing, 0, sizeof(int32_t), s));
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, f->n_e};
  const CertArgs a = cert_args(f);
  const int les = f->have_lesser ? 1 : 0;
  if (f->precision == ND_PREC_FP64)
    Kern<double>::selected(w, a, f->dt, x, y, count, les, Gr, Gl, Gg, n_missing, s);
  else if (f->precision == ND_PREC_MIXED)
    Kern<float>::selected(w, a, f->dt, x, y, count, les, Gr, Gl, Gg, n_missing, s);
  else
    Kern<DF>::selected(w, a, f->dt, x, y, count, les, Gr, Gl, Gg, n_missing, s);
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_contact_current(nd_fact* f, int32_t contact, double* current, double* current_im,
                                        void* stream) {
  if (!f || !current) return fail(ND_ERR_INVALID_ARG, "nd_contact_current: NULL argument");
  const nd_plan* p = f->plan;
  if (contact < 0 || contact >= p->n_contacts) return fail(ND_ERR_INVALID_ARG, "nd_contact_current: bad contact");
  if (f->n_e <= 0 || !f->have_lesser || !f->cur_sl || !f->cur_sg)
    return fail(ND_ERR_INVALID_ARG,
                "nd_contact_current: needs a preceding nd_diag_green with Sigma^< and Sigma^> (G^< or G^> requested)");
  cudaStream_t s = (cudaStream_t)stream;
  const int q = p->contact_cluster[contact];
  const ndgf::Cluster& c = p->cl[q];
  const int m = p->contact_ptr[contact + 1] - p->contact_ptr[contact];
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, f->n_e};
  double* dre = f->d_current;
  double* dim = f->d_current + f->n_e;
  const int ld = c.n + c.b;
  if (f->precision == ND_PREC_FP64)
    Kern<double>::current(w, c.off_P[0], c.off_P[1], ld, p->contact_row[contact], m, f->cur_sl, f->cur_sg,
                          p->sigma_elems, p->contact_soff[contact], dre, dim, s);
  else if (f->precision == ND_PREC_MIXED)
    Kern<float>::current(w, c.off_P[0], c.off_P[1], ld, p->contact_row[contact], m, f->cur_sl, f->cur_sg,
                         p->sigma_elems, p->contact_soff[contact], dre, dim, s);
  else
    Kern<DF>::current(w, c.off_P[0], c.off_P[1], ld, p->contact_row[contact], m, f->cur_sl, f->cur_sg,
                      p->sigma_elems, p->contact_soff[contact], dre, dim, s);
  ND_CUDA(cudaGetLastError());
  const size_t bytes = size_t(f->n_e) * sizeof(double);
  ND_CUDA(cudaMemcpyAsync(current, dre, bytes, is_device_ptr(current) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s));
  if (current_im)
    ND_CUDA(cudaMemcpyAsync(current_im, dim, bytes,
                            is_device_ptr(current_im) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return ND_OK;
}

// The two solves with the stored factorization behind nd_density_gradient
// (adjoint) and nd_density_jvp (forward): U = G^r E_C (unit right-hand sides
// at the contact sites; kept for the later calls on the same factorization),
// then G^r diag(c) conj(U) or G^r diag(c) U, and the contraction with Sigma^<.
template <typename T>
static nd_status adjoint_t(nd_fact* f, const double* c, double* t_out, bool forward, cudaStream_t s) {
  const nd_plan* p = f->plan;
  Work w{f->arena, f->se, f->aux, 2 * p->sigma_elems, f->n_e};
  const int M = p->adj_cols;
  nd_status st;
  auto solve = [&]() -> nd_status {
    nd_status r;
    if ((r = run_schedule<T>(f, f->sched_adj_fwd, f->tr_adj_fwd, w, nullptr, nullptr, s, 0,
                             &f->step_flops_adj_fwd)) != ND_OK)
      return r;
    return run_schedule<T>(f, f->sched_adj_bwd, f->tr_adj_bwd, w, nullptr, nullptr, s, 0, &f->step_flops_adj_bwd);
  };
  const bool cached = f->adj_u_valid;
  if (!cached) {
    Kern<T>::zero_range(w, f->adj_base, p->adj_elems, s);
    Kern<T>::adj_ones(w, f->d_ones, f->n_ones, s);
    if ((st = solve()) != ND_OK) return st;
  }
  Kern<T>::adj_mid(w, f->d_adj_desc, f->n_adj_desc, M, c, f->d_sites, f->dt, (forward ? 1 : 0) | (cached ? 2 : 0), s);
  if ((st = solve()) != ND_OK) return st;
  f->adj_u_valid = true;
  ContactTable ct{};
  ct.n = p->n_contacts;
  for (int k = 0; k < p->n_contacts; ++k) {
    ct.m[k] = p->contact_ptr[k + 1] - p->contact_ptr[k];
    ct.off[k] = p->contact_soff[k];
  }
  Kern<T>::adj_contract(w, f->d_adj_desc, f->n_adj_desc, M, ct, f->cur_sl, p->sigma_elems, f->d_sites, f->dt, t_out,
                        p->n, forward ? 1 : 0, s);
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

static nd_status adjoint_call(nd_fact* f, const double* c, double* t_out, bool forward, cudaStream_t s,
                              const char* name) {
  const std::string nm(name);
  if (!f || !c || !t_out) return fail(ND_ERR_INVALID_ARG, nm + ": NULL argument");
  const nd_plan* p = f->plan;
  if (!f->adj) return fail(ND_ERR_INVALID_ARG, nm + ": workspace created without ND_FACT_ADJOINT");
  if (f->n_e <= 0 || !f->have_lesser || !f->cur_sl)
    return fail(ND_ERR_INVALID_ARG, nm + ": needs a preceding nd_diag_green with Sigma^<");
  if (f->cur_pl) return fail(ND_ERR_UNSUPPORTED, nm + ": phonon Sigma^< is not supported");
  if (p->n_contacts < 1 || p->n_contacts > MAX_CONTACTS) return fail(ND_ERR_UNSUPPORTED, nm + ": needs 1 to 8 contacts");
  if (!is_device_ptr(t_out)) return fail(ND_ERR_INVALID_ARG, nm + ": t_out must be a device array");
  ND_CUDA(cudaMemcpyAsync(f->d_cvec, c, size_t(p->n) * sizeof(double),
                          is_device_ptr(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (f->precision == ND_PREC_FP64) return adjoint_t<double>(f, f->d_cvec, t_out, forward, s);
  if (f->precision == ND_PREC_MIXED) return adjoint_t<float>(f, f->d_cvec, t_out, forward, s);
  return adjoint_t<DF>(f, f->d_cvec, t_out, forward, s);
}

extern "C" nd_status nd_density_jvp(nd_fact* f, const double* v, double* t_out, void* stream) {
  return adjoint_call(f, v, t_out, true, (cudaStream_t)stream, "nd_density_jvp");
}

extern "C" nd_status nd_density_gradient(nd_fact* f, const double* c, double* t_out, void* stream) {
  return adjoint_call(f, c, t_out, false, (cudaStream_t)stream, "nd_density_gradient");
}

extern "C" nd_status nd_profile_launches(nd_fact* f, nd_launch_stats* out, int32_t max_out, int32_t* n_out) {
  if (!f || !n_out) return fail(ND_ERR_INVALID_ARG, "nd_profile_launches: NULL argument");
  ND_CUDA(cudaDeviceSynchronize());
  int cnt = 0;
  for (auto& r : f->prof.recs) {
    if (out && cnt < max_out) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      out[cnt] = nd_launch_stats{r.kind, r.count, r.max_dim, r.n_e, double(ms), r.flops};
    }
    ++cnt;
  }
  *n_out = cnt;
  return ND_OK;
}

extern "C" nd_status nd_profile(nd_fact* f, int32_t enable, nd_kernel_stats* stats, int32_t max_stats,
                                int32_t* n_stats) {
  if (!f) return fail(ND_ERR_INVALID_ARG, "nd_profile: NULL handle");
  int cnt = 0;
  if (stats && max_stats > 0) {
    ND_CUDA(cudaDeviceSynchronize());
    static const char* names[] = {"inverse",    "gemm",         "scatter",   "gather_sym", "gather_skew", "zero",
                                  "nph",        "gather_anc",   "scatter_rows", "colgather", "delay",     "loc",
                                  "gemm_tc",    "gemm_small",   "gemm_direct", "gemm_xl"};
    const int nk = int(sizeof(names) / sizeof(names[0]));
    std::vector<nd_kernel_stats> acc(nk);
    for (int k = 0; k < nk; ++k) {
      std::memset(&acc[k], 0, sizeof(nd_kernel_stats));
      std::strncpy(acc[k].name, names[k], sizeof(acc[k].name) - 1);
    }
    for (auto& r : f->prof.recs) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      if (r.kind < 0 || r.kind >= nk) continue;
      acc[r.kind].launches += 1;
      acc[r.kind].ms += ms;
      acc[r.kind].flops += r.flops;
      acc[r.kind].bytes += r.bytes;
    }
    for (int k = 0; k < nk && cnt < max_stats; ++k)
      if (acc[k].launches > 0) stats[cnt++] = acc[k];
  }
  if (n_stats) *n_stats = cnt;
  f->prof.clear();
  f->prof.on = enable != 0;
  return ND_OK;
}

extern "C" nd_status nd_density(const double* Gl, const double* weights, int32_t n_e, int32_t n, double scale,
                                int32_t accumulate, double* out, void* stream) {
  if (!Gl || !weights || !out || n_e <= 0 || n <= 0) return fail(ND_ERR_INVALID_ARG, "nd_density: bad argument");
  if (!is_device_ptr(Gl) || !is_device_ptr(weights) || !is_device_ptr(out))
    return fail(ND_ERR_INVALID_ARG, "nd_density: arrays must be device pointers");
  launch_density(Gl, weights, n_e, n, scale, accumulate, out, (cudaStream_t)stream);
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_fact_density(nd_fact* f, const double* weights, double scale, int32_t accumulate, double* out,
                                     void* stream) {
  if (!f || !weights || !out) return fail(ND_ERR_INVALID_ARG, "nd_fact_density: NULL argument");
  if (f->n_e <= 0 || !f->last_gl)
    return fail(ND_ERR_INVALID_ARG, "nd_fact_density: needs a preceding nd_diag_green that computed G^<");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = f->plan->n, n_e = f->n_e;
  const double* w = weights;
  if (!is_device_ptr(weights)) {
    ND_CUDA(cudaMemcpyAsync(f->d_w, weights, size_t(n_e) * sizeof(double), cudaMemcpyHostToDevice, s));
    w = f->d_w;
  }
  const bool out_dev = is_device_ptr(out);
  double* o = out_dev ? out : f->d_dens;
  if (!out_dev && accumulate)
    ND_CUDA(cudaMemcpyAsync(o, out, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
  launch_density(f->last_gl, w, n_e, n, scale, accumulate, o, s);
  ND_CUDA(cudaGetLastError());
  if (!out_dev) ND_CUDA(cudaMemcpyAsync(out, o, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s));
  return ND_OK;
}

extern "C" nd_status nd_autotune(nd_fact* f, const double* H_values, const double* sigma_r, const double* sigma_ph_r,
                                 const double* sigma_lesser, const double* sigma_greater, const double* ph_lesser,
                                 const double* ph_greater, const double* energies, int32_t n_e, double eta,
                                 int32_t reps, nd_tune_info* info, void* stream) {
  if (!f || reps < 1) return fail(ND_ERR_INVALID_ARG, "nd_autotune: bad argument");
  const nd_plan* p = f->plan;
  cudaStream_t s = (cudaStream_t)stream;
  const bool ph = (f->flags & ND_FACT_PHONON) != 0;
  const bool lesser = sigma_lesser || sigma_greater || ph_lesser || ph_greater;
  const std::vector<Step>* sched[4] = {&p->sched_factor, &p->sched_green, &p->sched_lesser[0], &p->sched_lesser[1]};
  const std::vector<TileRange>* trs[4] = {&f->tr_factor, &f->tr_green, &f->tr_lesser[0], &f->tr_lesser[1]};
  // candidate kernels per GEMM step: the default rules (-1), the large and the
  // small tile, the tensor cores (FP32 pairs, digit scratch within the limit),
  // one CTA per block (blocks up to 192) and the extra large tile
  auto allowed = [&](int q, int si, int c) {
    const Step& st = (*sched[q])[si];
    if (st.kind != ST_GEMM) return false;
    if (c == 2)
      return f->precision == ND_PREC_FP32X2 && (q != 3 || ph) && tc_scratch_fits(tc_step_scratch(st, f->gemm_all), f->max_ne);
    if (c == 3) return st.max_dim <= 192;
    if (c == 4) return st.max_dim > 32;  // the 64-row tiles only pay above the large tile's edge
    return true;
  };
  constexpr int NC = 5;  // candidates 0..4: large tile, small tile, tensor cores, one CTA per block, extra large tile
  std::array<std::vector<std::array<double, NC + 1>>, 4> ms;  // [schedule][step][candidate + 1]
  for (int q = 0; q < 4; ++q) ms[q].assign(sched[q]->size(), {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0});
  const bool prof_was = f->prof.on;
  nd_status st = ND_OK;
  int passes = 0;
  for (int c = -1; c < NC && st == ND_OK; ++c) {
    std::array<Choice, N_SCHED> forced;
    for (int q = 0; q < N_SCHED; ++q) {
      const size_t ns = q < 4 ? sched[q]->size() : (q == 4 ? f->sched_adj_fwd.size() : f->sched_adj_bwd.size());
      forced[q].assign(ns, -1);
      if (q < 4 && c >= 0)
        for (size_t si = 0; si < ns; ++si)
          if (allowed(q, int(si), c)) forced[q][si] = int8_t(c);
    }
    if ((st = build_all_tiles(f, &forced)) != ND_OK) break;
    for (int r = 0; r <= reps && st == ND_OK; ++r) {  // one untimed pass, then reps timed ones
      f->prof.clear();
      f->prof.on = r > 0;
      st = nd_factor(f, H_values, sigma_r, sigma_ph_r, energies, n_e, eta, stream);
      if (st == ND_OK)
        st = nd_diag_green(f, sigma_lesser, sigma_greater, ph_lesser, ph_greater, f->st_out[0],
                           lesser ? f->st_out[1] : nullptr, lesser ? f->st_out[2] : nullptr, stream);
      if (st != ND_OK) break;
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(ND_ERR_CUDA, "nd_autotune: a tuning pass failed");
        break;
      }
      if (r == 0) continue;
      for (auto& rec : f->prof.recs)
        for (int q = 0; q < 4; ++q)
          if (rec.tr == trs[q] && rec.si >= 0) {
            float t = 0.f;
            cudaEventElapsedTime(&t, rec.a, rec.b);
            const bool ok = c < 0 || forced[q][rec.si] == c;
            if (ok && (*sched[q])[rec.si].kind == ST_GEMM) {
              double& m = ms[q][rec.si][c + 1];
              m = m < 0.0 ? t / reps : m + t / reps;
            }
          }
    }
    ++passes;
  }
  f->prof.clear();
  f->prof.on = prof_was;
  if (st != ND_OK) {
    build_all_tiles(f, nullptr);
    return st;
  }
  // per step the fastest measured kernel
  std::array<Choice, N_SCHED> best;
  double t_def = 0.0, t_best = 0.0;
  int steps = 0, changed = 0, by_kind[5] = {0, 0, 0, 0, 0};
  for (int q = 0; q < N_SCHED; ++q) {
    const size_t ns = q < 4 ? sched[q]->size() : (q == 4 ? f->sched_adj_fwd.size() : f->sched_adj_bwd.size());
    best[q].assign(ns, -1);
    if (q >= 4) continue;
    for (size_t si = 0; si < ns; ++si) {
      if ((*sched[q])[si].kind != ST_GEMM) continue;
      const auto& m = ms[q][si];
      if (m[0] < 0.0) continue;  // not run (the phonon schedule without phonon inputs)
      int bc = -1;
      double bt = m[0];
      for (int c = 0; c < NC; ++c)
        if (m[c + 1] >= 0.0 && m[c + 1] < bt) {
          bt = m[c + 1];
          bc = c;
        }
      best[q][si] = int8_t(bc);
      ++steps;
      t_def += m[0];
      t_best += bt;
      if (bc >= 0) ++changed;
    }
  }
  if ((st = build_all_tiles(f, &best)) != ND_OK) return st;
  for (int q = 0; q < N_SCHED; ++q) f->choice[q] = best[q];
  for (int q = 0; q < 4; ++q)
    for (size_t si = 0; si < sched[q]->size(); ++si)
      if ((*sched[q])[si].kind == ST_GEMM && ms[q][si][0] >= 0.0) ++by_kind[(*trs[q])[si].kind];
  f->tuned = true;
  if (info) {
    info->ms_default = t_def;
    info->ms_tuned = t_best;
    info->gemm_steps = steps;
    info->changed = changed;
    info->passes = passes;
    for (int k = 0; k < 5; ++k) info->by_kind[k] = by_kind[k];
  }
  return ND_OK;
}

// The schedules whose GEMM steps carry a kernel choice, in the order of
// nd_fact_get_choice: fold, G^r, G^<, phonon G^<, adjoint forward and backward.
static std::array<const std::vector<Step>*, N_SCHED> choice_scheds(const nd_fact* f) {
  const nd_plan* p = f->plan;
  return {&p->sched_factor, &p->sched_green, &p->sched_lesser[0], &p->sched_lesser[1], &f->sched_adj_fwd,
          &f->sched_adj_bwd};
}

extern "C" nd_status nd_fact_get_choice(nd_fact* f, int8_t* choice, int32_t max, int32_t* n) {
  if (!f || !n || (choice && max < 0)) return fail(ND_ERR_INVALID_ARG, "nd_fact_get_choice: bad argument");
  const auto sc = choice_scheds(f);
  int64_t k = 0;
  for (int q = 0; q < N_SCHED; ++q)
    for (size_t si = 0; si < sc[q]->size(); ++si, ++k)
      if (choice && k < max) choice[k] = si < f->choice[q].size() ? f->choice[q][si] : int8_t(-1);
  *n = int32_t(k);
  if (choice && k > max) return fail(ND_ERR_INVALID_ARG, "nd_fact_get_choice: the array is too short");
  return ND_OK;
}

extern "C" nd_status nd_fact_set_choice(nd_fact* f, const int8_t* choice, int32_t n) {
  if (!f || !choice || n < 0) return fail(ND_ERR_INVALID_ARG, "nd_fact_set_choice: bad argument");
  const auto sc = choice_scheds(f);
  const bool ph = (f->flags & ND_FACT_PHONON) != 0;
  std::array<Choice, N_SCHED> want;
  int64_t k = 0;
  for (int q = 0; q < N_SCHED; ++q) {
    want[q].assign(sc[q]->size(), -1);
    for (size_t si = 0; si < sc[q]->size(); ++si, ++k) {
      if (k >= n) return fail(ND_ERR_INVALID_ARG, "nd_fact_set_choice: fewer entries than steps");
      const int c = choice[k];
      const Step& st = (*sc[q])[si];
      bool ok = c >= -1 && c <= 4 && (c == -1 || st.kind == ST_GEMM);
      if (ok && c == 2)
        ok = f->precision == ND_PREC_FP32X2 && (q != 3 || ph) && tc_scratch_fits(tc_step_scratch(st, f->gemm_all), f->max_ne);
      if (ok && c == 3) ok = st.max_dim <= 192;
      if (ok && c == 4) ok = st.max_dim > 32;
      if (!ok) return fail(ND_ERR_INVALID_ARG, "nd_fact_set_choice: a kernel that this step cannot take");
      want[q][si] = int8_t(c);
    }
  }
  if (k != n) return fail(ND_ERR_INVALID_ARG, "nd_fact_set_choice: more entries than steps");
  nd_status st = build_all_tiles(f, &want);
  if (st != ND_OK) return st;
  f->choice = want;
  return ND_OK;
}

extern "C" nd_status nd_fact_set_wait_limit(nd_fact* f, int64_t polls) {
  if (!f || polls < 0) return fail(ND_ERR_INVALID_ARG, "nd_fact_set_wait_limit: bad argument");
  f->tc_wait_polls = polls;
  f->clear_graphs();  // the recorded launches carry the old limit
  return ND_OK;
}

extern "C" nd_status nd_fact_status(nd_fact* f, int32_t* n_singular) {
  if (!f) return fail(ND_ERR_INVALID_ARG, "nd_fact_status: NULL handle");
  int h = 0, to = 0, ie[2] = {0, 0};
  ND_CUDA(cudaMemcpy(&h, f->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  ND_CUDA(cudaMemcpy(&to, f->d_tc_timeout, sizeof(int), cudaMemcpyDeviceToHost));
  ND_CUDA(cudaMemcpy(ie, f->d_inerr, sizeof(ie), cudaMemcpyDeviceToHost));
  if (n_singular) *n_singular = h;
  if (to) return fail(ND_ERR_TIMEOUT, "nd_fact_status: a tensor-core product gave up waiting; results are invalid");
  if (ie[0])
    return fail(ND_ERR_NOT_SYMMETRIC,
                "nd_fact_status: the device H values or Sigma^r blocks of the last nd_factor are not (complex) "
                "symmetric or not finite; results are invalid");
  if (ie[1])
    return fail(ND_ERR_NOT_SKEW_HERMITIAN,
                "nd_fact_status: the device Sigma^< / Sigma^> of the last nd_diag_green are not skew-Hermitian or "
                "not finite; G^< / G^> are invalid");
  if (h > 0) return fail(ND_ERR_SINGULAR, "nd_fact_status: " + std::to_string(h) + " singular pivot(s)");
  return ND_OK;
}

// ---------------------------------------------------------------------------
// Leads (S1a)

namespace {
// Cyclic Jacobi eigen-decomposition of a real symmetric matrix (row major);
// on return A is diagonal (eigenvalues) and V holds the eigenvectors in
// its columns.  Golub & Van Loan, Matrix Computations, Sec. 8.5.
void jacobi_eig(int m, std::vector<double>& A, std::vector<double>& V) {
  V.assign(size_t(m) * m, 0.0);
  for (int i = 0; i < m; ++i) V[size_t(i) * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double a = A[size_t(i) * m + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[size_t(p) * m + q];
        if (apq == 0.0) continue;
        const double app = A[size_t(p) * m + p], aqq = A[size_t(q) * m + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[size_t(k) * m + p], akq = A[size_t(k) * m + q];
          A[size_t(k) * m + p] = c * akp - s * akq;
          A[size_t(k) * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[size_t(p) * m + k], aqk = A[size_t(q) * m + k];
          A[size_t(p) * m + k] = c * apk - s * aqk;
          A[size_t(q) * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[size_t(k) * m + p], vkq = V[size_t(k) * m + q];
          V[size_t(k) * m + p] = c * vkp - s * vkq;
          V[size_t(k) * m + q] = s * vkp + c * vkq;
        }
      }
  }
}
}  // namespace

struct nd_lead {
  int m = 0, m_c = 0;
  bool modes = false;
  double hop = 0.0;
  double *d_U = nullptr, *d_eps = nullptr;  // transverse modes (uniform lead)
  // decimation (general lead): H00, H01, tau on the device, workspace grown on demand
  double *d_H00 = nullptr, *d_H01 = nullptr, *d_tau = nullptr, *d_work = nullptr;
  int* d_status = nullptr;  // [0] energies not converged, [1] singular pivots
  double scale = 1.0;
  int64_t work_energies = 0;
  cudaStream_t last_stream = nullptr;
  ~nd_lead() {
    cudaFree(d_U);
    cudaFree(d_eps);
    cudaFree(d_H00);
    cudaFree(d_H01);
    cudaFree(d_tau);
    cudaFree(d_work);
    cudaFree(d_status);
  }
};

constexpr int LEAD_MAX_ITER = 100;
constexpr double LEAD_TOL = 1e-14;

extern "C" nd_status nd_lead_create(int32_t m, int32_t m_c, const double* H00, const double* H01, const double* tau,
                                    nd_lead** out) {
  if (!out || !H00 || !H01 || !tau || m <= 0 || m_c <= 0) return fail(ND_ERR_INVALID_ARG, "nd_lead_create: bad argument");
  *out = nullptr;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      if (std::fabs(H00[size_t(i) * m + j] - H00[size_t(j) * m + i]) > 1e-12 * (1.0 + std::fabs(H00[size_t(i) * m + j])))
        return fail(ND_ERR_NOT_SYMMETRIC, "nd_lead_create: H00 not symmetric");
  // H01 = -h I and tau = -h I ?
  const double h = -H01[0];
  bool uniform = (m == m_c) && h != 0.0;
  for (int i = 0; i < m && uniform; ++i)
    for (int j = 0; j < m && uniform; ++j) {
      const double want = (i == j) ? -h : 0.0;
      uniform = std::fabs(H01[size_t(i) * m + j] - want) <= 1e-14 * std::fabs(h) &&
                std::fabs(tau[size_t(i) * m + j] - want) <= 1e-14 * std::fabs(h);
    }
  auto L = new nd_lead();
  L->m = m;
  L->m_c = m_c;
  if (!uniform) {
    std::vector<double> h00(H00, H00 + size_t(m) * m), h01(H01, H01 + size_t(m) * m), t(tau, tau + size_t(m_c) * m);
    for (double v : h00) L->scale = std::max(L->scale, std::fabs(v));
    for (double v : h01) L->scale = std::max(L->scale, std::fabs(v));
    if (upload(h00, &L->d_H00) != ND_OK || upload(h01, &L->d_H01) != ND_OK || upload(t, &L->d_tau) != ND_OK ||
        cudaMalloc(&L->d_status, 2 * sizeof(int)) != cudaSuccess || cudaMemset(L->d_status, 0, 2 * sizeof(int)) != cudaSuccess) {
      delete L;
      return fail(ND_ERR_OOM, "nd_lead_create: device allocation failed");
    }
    *out = L;
    return ND_OK;
  }
  L->modes = true;
  L->hop = h;
  std::vector<double> A(H00, H00 + size_t(m) * m), V;
  jacobi_eig(m, A, V);
  std::vector<double> eps(m);
  for (int i = 0; i < m; ++i) eps[i] = A[size_t(i) * m + i];
  if (upload(V, &L->d_U) != ND_OK || upload(eps, &L->d_eps) != ND_OK) {
    delete L;
    return ND_ERR_OOM;
  }
  *out = L;
  return ND_OK;
}

extern "C" nd_status nd_lead_sigma(nd_lead* L, const double* energies, int32_t n_e, double eta, double* sigma_out,
                                   int64_t stride, int64_t offset, void* stream) {
  if (!L || !energies || !sigma_out || n_e <= 0) return fail(ND_ERR_INVALID_ARG, "nd_lead_sigma: bad argument");
  if (!is_device_ptr(energies) || !is_device_ptr(sigma_out))
    return fail(ND_ERR_INVALID_ARG, "nd_lead_sigma: energies and sigma_out must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  L->last_stream = st;
  if (L->modes) {
    launch_lead_modes(L->d_U, L->d_eps, L->m, L->hop, energies, n_e, eta, sigma_out, stride, offset, st);
  } else {
    if (n_e > L->work_energies) {
      cudaFree(L->d_work);
      L->d_work = nullptr;
      L->work_energies = 0;
      const size_t bytes = lead_decimation_work_elems(L->m, L->m_c) * size_t(n_e) * sizeof(double2);
      if (cudaMalloc(&L->d_work, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ND_ERR_OOM, "nd_lead_sigma: cannot allocate the decimation workspace");
      }
      L->work_energies = n_e;
    }
    launch_lead_decimation(L->d_H00, L->d_H01, L->d_tau, L->m, L->m_c, energies, n_e, eta, L->scale, LEAD_TOL,
                           LEAD_MAX_ITER, sigma_out, stride, offset, L->d_work, L->d_status, st);
  }
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_lead_status(nd_lead* L, int32_t* n_unconverged, int32_t* n_singular) {
  if (!L || !n_unconverged || !n_singular) return fail(ND_ERR_INVALID_ARG, "nd_lead_status: bad argument");
  *n_unconverged = 0;
  *n_singular = 0;
  if (L->modes) return ND_OK;
  int h[2] = {0, 0};
  ND_CUDA(cudaStreamSynchronize(L->last_stream));
  ND_CUDA(cudaMemcpy(h, L->d_status, sizeof(h), cudaMemcpyDeviceToHost));
  ND_CUDA(cudaMemset(L->d_status, 0, sizeof(h)));
  *n_unconverged = h[0];
  *n_singular = h[1];
  return (h[0] || h[1]) ? fail(ND_ERR_SINGULAR, "nd_lead_status: decimation did not converge or met a zero pivot")
                        : ND_OK;
}

extern "C" void nd_lead_destroy(nd_lead* L) { delete L; }

extern "C" nd_status nd_sigma_lesser_fermi(const double* sigma_r, int32_t n_e, int32_t n_contacts, const int32_t* m_c,
                                           const double* mu, double kT, const double* energies, double* sigma_lesser,
                                           double* sigma_greater, void* stream) {
  if (!sigma_r || !m_c || !mu || !energies || n_e <= 0 || n_contacts <= 0 || !(kT > 0))
    return fail(ND_ERR_INVALID_ARG, "nd_sigma_lesser_fermi: bad argument");
  std::vector<int64_t> off(n_contacts + 1, 0);
  for (int c = 0; c < n_contacts; ++c) {
    if (m_c[c] <= 0) return fail(ND_ERR_INVALID_ARG, "nd_sigma_lesser_fermi: contact size must be positive");
    off[c + 1] = off[c] + int64_t(m_c[c]) * m_c[c];
  }
  // contacts in groups of MAX_CONTACTS per launch, each with its offset in the packed arrays
  for (int c0 = 0; c0 < n_contacts; c0 += MAX_CONTACTS) {
    ContactTable ct{};
    ct.n = std::min(MAX_CONTACTS, n_contacts - c0);
    for (int j = 0; j < ct.n; ++j) {
      ct.m[j] = m_c[c0 + j];
      ct.off[j] = off[c0 + j];
      ct.mu[j] = mu[c0 + j];
    }
    launch_sigma_lesser(sigma_r, n_e, ct, kT, energies, off[n_contacts], sigma_lesser, sigma_greater,
                        (cudaStream_t)stream);
  }
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_phonon_scba(int32_t n, int32_t n_e, double D, double mix, const double* Gr, const double* Gl,
                                    const double* Gg, double* ph_r, double* ph_lesser, double* ph_greater,
                                    double* stats, void* stream) {
  if (n <= 0 || n_e <= 0 || !Gr || !Gl || !Gg || !ph_r || !ph_lesser || !ph_greater || !stats)
    return fail(ND_ERR_INVALID_ARG, "nd_phonon_scba: bad argument");
  if (!(D >= 0.0) || !(mix > 0.0 && mix <= 1.0))
    return fail(ND_ERR_INVALID_ARG, "nd_phonon_scba: need D >= 0 and 0 < mix <= 1");
  const void* ptrs[7] = {Gr, Gl, Gg, ph_r, ph_lesser, ph_greater, stats};
  for (const void* q : ptrs)
    if (!is_device_ptr(q)) return fail(ND_ERR_INVALID_ARG, "nd_phonon_scba: arrays must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  ND_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(double), s));
  launch_phonon_scba(n, n_e, D, mix, Gr, Gl, Gg, ph_r, ph_lesser, ph_greater, stats, s);
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}

extern "C" nd_status nd_phonon_const(int32_t n, int32_t n_e, double gamma, double mu, double kT,
                                     const double* energies, double* ph_r, double* ph_lesser, double* ph_greater,
                                     void* stream) {
  if (n <= 0 || n_e <= 0 || !energies || !(kT > 0)) return fail(ND_ERR_INVALID_ARG, "nd_phonon_const: bad argument");
  launch_phonon(n, n_e, gamma, mu, kT, energies, ph_r, ph_lesser, ph_greater, (cudaStream_t)stream);
  ND_CUDA(cudaGetLastError());
  return ND_OK;
}
