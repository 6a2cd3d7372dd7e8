// Launch schedule of the numeric phases, built once per plan on the host.
//
// Every step is one batched launch over (clusters of one tree level) x
// (energies).  Descriptors hold per-energy workspace offsets; the kernels add
// energy * (workspace elements per energy).  Cluster regions (see Cluster):
//   F   = [A_ii | A_iB]  -> A_ii^{-1} in place after the fold
//   Psi = -A_ii^{-1} A_iB
//   BB  = Schur update accumulator (fold), then G_BB (extraction)
//   G   = [G_II | G_IB]
//   P_s = [P_II | P_IB], PBB_s = P_BB, for s = 0 (Sigma^<, G^<) and s = 1 (Sigma^>, G^>)
//   and, on clusters whose N row block is nonzero, the ancestor-column blocks
//   GX = G_{I,anc}, NX_s = N_{I, I+anc}, NB_s = N_{B,anc}, PX_s = A_ii^{-1} NX_s.

#include <algorithm>
#include <unordered_map>

#include "nd_internal.h"

namespace ndgf {

namespace {

struct Builder {
  nd_plan* p;
  std::vector<Step>* cur = nullptr;
  Step st{};

  void begin(std::vector<Step>* sched, int kind) {
    cur = sched;
    st = Step{kind, 0, 0, 0};
    switch (kind) {
      case ST_INVERSE: st.begin = int32_t(p->inv_desc.size()); break;
      case ST_GEMM: st.begin = int32_t(p->gemm_desc.size()); break;
      case ST_SCATTER: st.begin = int32_t(p->scat_desc.size()); break;
      case ST_GATHER_SYM:
      case ST_GATHER_SKEW: st.begin = int32_t(p->gath_desc.size()); break;
      case ST_ZERO: st.begin = int32_t(p->zero_desc.size()); break;
      case ST_NPH: st.begin = int32_t(p->nph_desc.size()); break;
      case ST_GATHER_ANC: st.begin = int32_t(p->anc_desc.size()); break;
      case ST_SCATTER_ROWS: st.begin = int32_t(p->rows_desc.size()); break;
      case ST_COLGATHER: st.begin = int32_t(p->colg_desc.size()); break;
      case ST_DELAY: st.begin = int32_t(p->delay_desc.size()); break;
      case ST_LOC: st.begin = int32_t(p->loc_desc.size()); break;
    }
  }
  void end() {
    int32_t e = 0;
    switch (st.kind) {
      case ST_INVERSE: e = int32_t(p->inv_desc.size()); break;
      case ST_GEMM: e = int32_t(p->gemm_desc.size()); break;
      case ST_SCATTER: e = int32_t(p->scat_desc.size()); break;
      case ST_GATHER_SYM:
      case ST_GATHER_SKEW: e = int32_t(p->gath_desc.size()); break;
      case ST_ZERO: e = int32_t(p->zero_desc.size()); break;
      case ST_NPH: e = int32_t(p->nph_desc.size()); break;
      case ST_GATHER_ANC: e = int32_t(p->anc_desc.size()); break;
      case ST_SCATTER_ROWS: e = int32_t(p->rows_desc.size()); break;
      case ST_COLGATHER: e = int32_t(p->colg_desc.size()); break;
      case ST_DELAY: e = int32_t(p->delay_desc.size()); break;
      case ST_LOC: e = int32_t(p->loc_desc.size()); break;
    }
    st.count = e - st.begin;
    if (st.count > 0) cur->push_back(st);
  }
  void dim(int d) { st.max_dim = std::max(st.max_dim, d); }

  void gemm(int64_t C, int ldc, int64_t D, int ldd, int64_t A, int lda, int opA, int64_t B, int ldb, int opB,
            int m, int n, int k, double alpha, double beta) {
    if (m <= 0 || n <= 0) return;
    GemmDesc g{};
    g.offA = A; g.offB = B; g.offC = C; g.offD = D;
    g.m = m; g.n = n; g.k = k;
    g.lda = lda; g.ldb = ldb; g.ldc = ldc; g.ldd = ldd;
    g.opA = opA; g.opB = opB;
    g.alpha = alpha; g.beta = beta;
    p->gemm_desc.push_back(g);
    dim(std::max(m, std::max(n, k)));
  }
};

}  // namespace

namespace {

// Size class of a block edge: launches of one class share a CTA shape.
int size_class(int d) { return d <= 24 ? 0 : d <= 48 ? 1 : d <= 96 ? 2 : d <= 192 ? 3 : 4; }

// Every inverse, delay and GEMM step of a schedule becomes one launch per size
// class of its blocks (descriptors reordered inside the step's range), so
// that a few large blocks (the contact leaves, say) do not set the CTA shape,
// shared memory and tile of thousands of small ones.
template <typename D, typename Dim>
void split_kind(std::vector<Step>& sched, int kind, std::vector<D>& table, Dim dim) {
  std::vector<Step> out;
  for (const Step& st : sched) {
    if (st.kind != kind || st.count <= 1) {
      out.push_back(st);
      continue;
    }
    std::vector<D> part(table.begin() + st.begin, table.begin() + st.begin + st.count);
    std::stable_sort(part.begin(), part.end(),
                     [&](const D& a, const D& b) { return size_class(dim(a)) < size_class(dim(b)); });
    std::copy(part.begin(), part.end(), table.begin() + st.begin);
    int i = 0;
    while (i < st.count) {
      const int cls = size_class(dim(part[i]));
      int j = i, md = 0;
      while (j < st.count && size_class(dim(part[j])) == cls) md = std::max(md, dim(part[j++]));
      out.push_back(Step{st.kind, st.begin + i, j - i, md});
      i = j;
    }
  }
  sched = std::move(out);
}

void split_by_size(nd_plan* p, std::vector<Step>& sched) {
  split_kind(sched, ST_INVERSE, p->inv_desc, [](const InvDesc& d) { return d.n; });
  split_kind(sched, ST_DELAY, p->delay_desc, [](const DelayDesc& d) { return d.nf; });
  split_kind(sched, ST_GEMM, p->gemm_desc, [](const GemmDesc& g) { return std::max(g.m, std::max(g.n, g.k)); });
}

}  // namespace

void build_schedules(nd_plan* p) {
  auto& cl = p->cl;
  const int nc = int(cl.size());
  // transpose index of every CSR entry (the pattern is structurally symmetric)
  {
    std::vector<std::pair<int32_t, int32_t>> byc(p->nnz);  // (column, CSR index), sorted per row
    for (int r = 0; r < p->n; ++r) {
      for (int q = p->rowptr[r]; q < p->rowptr[r + 1]; ++q) byc[q] = {p->colind[q], q};
      std::sort(byc.begin() + p->rowptr[r], byc.begin() + p->rowptr[r + 1]);
    }
    p->csr_T.assign(p->nnz, -1);
    for (int r = 0; r < p->n; ++r)
      for (int q = p->rowptr[r]; q < p->rowptr[r + 1]; ++q) {
        const int c = p->colind[q];
        auto it = std::lower_bound(byc.begin() + p->rowptr[c], byc.begin() + p->rowptr[c + 1],
                                   std::make_pair(int32_t(r), int32_t(-1)));
        p->csr_T[q] = it->second;  // present: nd_analyze checked the pattern's symmetry
      }
  }
  std::vector<int32_t> site_begin(nc), map_begin(nc);
  p->root_scratch_elems = 0;
  p->unk_q.clear();
  p->unk_r.clear();
  for (int i = 0; i < nc; ++i) {
    site_begin[i] = int32_t(p->sites.size());
    p->sites.insert(p->sites.end(), cl[i].I.begin(), cl[i].I.end());
    for (int r = 0; r < cl[i].nf(); ++r) {
      p->unk_q.push_back(i);
      p->unk_r.push_back(r);
    }
    map_begin[i] = int32_t(p->maps.size());
    p->maps.insert(p->maps.end(), cl[i].map.begin(), cl[i].map.end());
  }
  p->n_unk = int64_t(p->sites.size());
  // contact offsets in the packed Sigma arrays
  std::vector<int32_t> soff(p->n_contacts + 1, 0);
  for (int c = 0; c < p->n_contacts; ++c) {
    int m = p->contact_ptr[c + 1] - p->contact_ptr[c];
    soff[c + 1] = soff[c] + m * m;
  }
  p->contact_cluster.assign(p->n_contacts, -1);
  p->contact_row.assign(p->n_contacts, 0);
  p->contact_soff.assign(p->n_contacts, 0);
  for (int c = 0; c < p->n_contacts; ++c) p->contact_soff[c] = soff[c];
  for (int i = 0; i < nc; ++i)
    for (auto& ct : cl[i].contacts) {
      p->contact_cluster[ct.first] = i;
      p->contact_row[ct.first] = ct.second;
    }
  // ---- S1 assembly lists ----------------------------------------------------
  {
    std::vector<int> posB(p->n + p->n_virtual, -1);
    for (int i = 0; i < nc; ++i) {
      Cluster& c = cl[i];
      const int ld = c.n + c.b;
      for (int k = 0; k < c.b; ++k) posB[c.B[k]] = k;
      AssembleDesc a{};
      a.off_F = c.off_F;
      a.off_BB = c.off_BB;
      a.n = c.nf();
      a.n_own = c.n_own;
      a.b = c.b;
      a.ld = ld;
      a.site_begin = site_begin[i];
      a.ent_begin = int32_t(p->ent_dst.size());
      for (int r = 0; r < c.n_own; ++r) {
        const int v = c.I[r];
        for (int q = p->rowptr[v]; q < p->rowptr[v + 1]; ++q) {
          const int u = p->colind[q];
          int dst = -1;
          if (p->owner[u] == i)
            dst = r * ld + p->pos[u];
          else if (posB[u] >= 0)
            dst = r * ld + c.n + posB[u];
          if (dst >= 0) {
            p->ent_dst.push_back(dst);
            p->ent_src.push_back(q);
          }
        }
      }
      a.ent_end = int32_t(p->ent_dst.size());
      a.c0 = a.m0 = a.soff0 = a.c1 = a.m1 = a.soff1 = 0;
      if (!c.contacts.empty()) {
        int cid = c.contacts[0].first;
        a.c0 = c.contacts[0].second;
        a.m0 = p->contact_ptr[cid + 1] - p->contact_ptr[cid];
        a.soff0 = soff[cid];
      }
      if (c.contacts.size() > 1) {
        int cid = c.contacts[1].first;
        a.c1 = c.contacts[1].second;
        a.m1 = p->contact_ptr[cid + 1] - p->contact_ptr[cid];
        a.soff1 = soff[cid];
      }
      p->asm_desc.push_back(a);
      for (int k = 0; k < c.b; ++k) posB[c.B[k]] = -1;
    }
  }
  std::vector<std::vector<int>> lev(p->n_levels + 1);
  for (int i = 0; i < nc; ++i) lev[cl[i].level].push_back(i);
  int max_slot = 0;
  for (int i = 0; i < nc; ++i) max_slot = std::max(max_slot, cl[i].slot);

  Builder B{p};
  // ---- S2/S3 fold: for l = 1..L, invert A_ii; Psi; Schur update; extend-add
  for (int l = 1; l <= p->n_levels; ++l) {
    B.begin(&p->sched_factor, ST_DELAY);  // delayed pivots: choose, reorder the front
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.k == 0) continue;
      p->delay_desc.push_back(DelayDesc{c.off_F, c.off_BB, c.off_G, c.nf(), c.k, c.n + c.b, c.b, site_begin[i],
                                        site_begin[c.parent], c.dslot});
      B.dim(c.nf());
    }
    B.end();
    B.begin(&p->sched_factor, ST_INVERSE);
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      // roots are inverted in complex128 on the single-precision paths, each in
      // its own scratch region (several roots share a launch in a batch of devices)
      int64_t scr = 0;
      if (c.b == 0) {
        scr = p->root_scratch_elems;
        p->root_scratch_elems += int64_t(c.n) * c.n;
      }
      p->inv_desc.push_back(InvDesc{c.off_F, c.n, c.n + c.b, i, c.b == 0 ? 1 : 0, scr});
      B.dim(c.n);
    }
    B.end();
    B.begin(&p->sched_factor, ST_GEMM);  // Psi = -A_ii^{-1} A_iB
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const int ld = c.n + c.b;
      B.gemm(c.off_Psi, c.b, c.off_Psi, c.b, c.off_F, ld, OP_N, c.off_F + c.n, ld, OP_N, c.n, c.b, c.n, -1.0, 0.0);
    }
    B.end();
    B.begin(&p->sched_factor, ST_GEMM);  // U = A_BB-updates + A_iB^T Psi
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const int ld = c.n + c.b;
      B.gemm(c.off_BB, c.b, c.off_BB, c.b, c.off_F + c.n, ld, OP_T, c.off_Psi, c.b, OP_N, c.b, c.b, c.n, 1.0, 1.0);
    }
    B.end();
    for (int s = 0; s <= max_slot; ++s) {
      B.begin(&p->sched_factor, ST_SCATTER);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0 || c.slot != s) continue;
        const Cluster& P = cl[c.parent];
        p->scat_desc.push_back(ScatterDesc{c.off_BB, P.off_F, P.off_BB, c.b, P.n, P.b, map_begin[i], P.k});
        B.dim(c.b);
      }
      B.end();
    }
  }
  // final position of every front row once all delayed pivots are chosen
  // (top down: a delayed row ends where its parent's virtual row ends)
  if (p->n_virtual > 0)
    for (int l = p->n_levels; l >= 1; --l) {
      B.begin(&p->sched_factor, ST_LOC);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        p->loc_desc.push_back(LocDesc{site_begin[i], c.nf(), c.n, i, c.parent >= 0 ? site_begin[c.parent] : -1,
                                      c.dslot});
        B.dim(c.nf());
      }
      B.end();
    }
  // ---- S4 G^r extraction -----------------------------------------------------
  B.begin(&p->sched_green, ST_GEMM);  // clusters without boundary: G_II = A_ii^{-1}
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = cl[i];
    if (c.b != 0) continue;
    B.gemm(c.off_G, c.n, c.off_F, c.n, 0, 1, OP_N, 0, 1, OP_N, c.n, c.n, 0, 0.0, 1.0);
  }
  B.end();
  for (int l = p->n_levels; l >= 1; --l) {
    B.begin(&p->sched_green, ST_GATHER_SYM);
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const Cluster& P = cl[c.parent];
      p->gath_desc.push_back(GatherDesc{c.off_BB, P.off_G, P.off_BB, c.b, P.n, P.b, map_begin[i], P.k,
                                        site_begin[c.parent]});
      B.dim(c.b);
    }
    B.end();
    B.begin(&p->sched_green, ST_GEMM);  // G_IB = Psi G_BB
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const int ld = c.n + c.b;
      B.gemm(c.off_G + c.n, ld, c.off_G + c.n, ld, c.off_Psi, c.b, OP_N, c.off_BB, c.b, OP_N, c.n, c.b, c.b, 1.0, 0.0);
    }
    B.end();
    B.begin(&p->sched_green, ST_GEMM);  // G_II = A_ii^{-1} + Psi G_IB^T
    for (int i : lev[l]) {
      const Cluster& c = cl[i];
      if (c.b == 0) continue;
      const int ld = c.n + c.b;
      B.gemm(c.off_G, ld, c.off_F, ld, c.off_Psi, c.b, OP_N, c.off_G + c.n, ld, OP_T, c.n, c.n, c.b, 1.0, 1.0);
    }
    B.end();
  }
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = cl[i];
    p->diag_g.push_back(DiagDesc{c.off_G, c.n, c.n + c.b, site_begin[i]});
    for (int s = 0; s < 2; ++s) p->diag_p[s].push_back(DiagDesc{c.off_P[s], c.n, c.n + c.b, site_begin[i]});
  }
  // ---- S5-S8 G^< and G^> -----------------------------------------------------
  // Paper Sec. 3.2: N = Sigma^< (G^(0))^dagger uses G^(0)_{ij} for every
  // ancestor cluster j of i, so a cluster whose row block of N is nonzero
  // carries N over I_i and all ancestor sites (Y_i); its fold update moves
  // up row by row.  The P extraction only needs [P_II | P_IB] and P_BB.
  std::vector<int32_t> bsite_begin(nc), anc_begin(nc), cmap_begin(nc);
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = cl[i];
    bsite_begin[i] = int32_t(p->site_ids.size());
    for (int u : c.B) p->site_ids.push_back(site_begin[p->owner[u]] + p->pos[u]);
    anc_begin[i] = int32_t(p->anc_q.size());
    for (int a = c.parent; a >= 0; a = cl[a].parent)
      for (int r = 0; r < cl[a].n; ++r) {
        p->anc_q.push_back(a);
        p->anc_r.push_back(r);
      }
    cmap_begin[i] = int32_t(p->cmaps.size());
    for (int k = 0; k < c.b; ++k) {
      const int u = c.B[k], o = p->owner[u];
      p->cmaps.push_back(c.n + c.A - cl[o].n - cl[o].A + p->pos[u]);
    }
    p->cl_n.push_back(c.n);
    p->cl_A.push_back(c.A);
    p->cl_ldG.push_back(c.n + c.b);
    p->cl_offG.push_back(c.off_G);
    p->cl_offGX[0].push_back(c.ext[0].off_GX);
    p->cl_offGX[1].push_back(c.ext[1].off_GX);
    p->cl_offP[0].push_back(c.off_P[0]);
    p->cl_offP[1].push_back(c.off_P[1]);
  }
  // ---- S9 certificate term lists --------------------------------------------
  for (int i = 0; i < nc; ++i)
    if (cl[i].b) p->psi_desc.push_back(ZeroDesc{cl[i].off_Psi, int64_t(cl[i].n) * cl[i].b});
  // Where each entry X_kj of a coupled pair is stored is decided at run time
  // (the rows a cluster eliminates are per energy with delayed pivots): the
  // static part is the slot of every site, each cluster's front geometry and
  // its boundary slots sorted for a binary search.
  p->cert_cl.clear();
  p->cert_bslot.clear();
  p->cert_bidx.clear();
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = cl[i];
    CertCluster cc{};
    cc.offG = c.off_G;
    cc.offP = c.off_P[0];
    cc.offPg = c.off_P[1];
    cc.sb = site_begin[i];
    cc.n = c.n;
    cc.ld = c.n + c.b;
    cc.parent = c.parent;
    cc.dslot = c.parent >= 0 ? c.dslot : -1;
    cc.first_desc = c.first_desc;
    cc.bs = int32_t(p->cert_bslot.size());
    cc.b = c.b;
    std::vector<std::pair<int32_t, int32_t>> sl(c.b);
    for (int k = 0; k < c.b; ++k) sl[k] = {p->site_ids[bsite_begin[i] + k], k};
    std::sort(sl.begin(), sl.end());
    for (auto& x : sl) {
      p->cert_bslot.push_back(x.first);
      p->cert_bidx.push_back(x.second);
    }
    p->cert_cl.push_back(cc);
  }
  p->cert_slot.assign(p->n, 0);
  for (int j = 0; j < p->n; ++j) p->cert_slot[j] = site_begin[p->owner[j]] + p->pos[j];
  {
    std::vector<int32_t> contact_of(p->n, -1), cpos(p->n, -1);
    for (int c = 0; c < p->n_contacts; ++c)
      for (int q = p->contact_ptr[c]; q < p->contact_ptr[c + 1]; ++q) {
        contact_of[p->contact_idx[q]] = c;
        cpos[p->contact_idx[q]] = q - p->contact_ptr[c];
      }
    p->cert_ptr.assign(1, 0);
    p->cert_nb.clear();
    p->cert_coef.clear();
    for (int j = 0; j < p->n; ++j) {
      for (int q = p->rowptr[j]; q < p->rowptr[j + 1]; ++q) {
        p->cert_nb.push_back(p->colind[q]);
        p->cert_coef.push_back(q);
      }
      const int ct = contact_of[j];
      if (ct >= 0) {
        const int m = p->contact_ptr[ct + 1] - p->contact_ptr[ct];
        for (int q = p->contact_ptr[ct]; q < p->contact_ptr[ct + 1]; ++q) {
          p->cert_nb.push_back(p->contact_idx[q]);
          p->cert_coef.push_back(-1 - int32_t(soff[ct] + cpos[j] * m + (q - p->contact_ptr[ct])));
        }
      }
      p->cert_ptr.push_back(int32_t(p->cert_nb.size()));
    }
  }
  for (int v = 0; v < 2; ++v) {
    auto* S = &p->sched_lesser[v];
    auto active = [&](int i) { return v == 1 || cl[i].nactive; };
    B.begin(S, ST_ZERO);
    for (int i = 0; i < nc; ++i) {
      const Cluster& c = cl[i];
      const auto& x = c.ext[v];
      for (int s = 0; s < 2; ++s) {
        if (active(i)) {
          if (v == 0) p->zero_desc.push_back(ZeroDesc{x.off_NX[s], int64_t(c.n) * (c.n + c.A)});
          if (c.b && c.A) p->zero_desc.push_back(ZeroDesc{x.off_NB[s], int64_t(c.b) * c.A});
        } else if (c.b == 0) {
          p->zero_desc.push_back(ZeroDesc{c.off_P[s], int64_t(c.n) * c.n});
        }
      }
    }
    B.end();
    for (int l = p->n_levels; l >= 1; --l) {  // G_{I,anc} = Psi G_{B,anc}, top down
      B.begin(S, ST_GATHER_ANC);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (!active(i) || c.b == 0 || c.A == 0) continue;
        p->anc_desc.push_back(AncGatherDesc{c.ext[v].off_GBA, c.b, c.A, bsite_begin[i], anc_begin[i]});
        B.dim(c.b);
      }
      B.end();
      B.begin(S, ST_GEMM);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (!active(i) || c.b == 0 || c.A == 0) continue;
        B.gemm(c.ext[v].off_GX, c.A, c.ext[v].off_GX, c.A, c.off_Psi, c.b, OP_N, c.ext[v].off_GBA, c.A, OP_N, c.n, c.A,
               c.b, 1.0, 0.0);
      }
      B.end();
    }
    if (v == 1) {
      B.begin(S, ST_NPH);  // N = Sigma_ph conj(G_{I,Y}) on every cluster
      for (int i = 0; i < nc; ++i) {
        const Cluster& c = cl[i];
        for (int s = 0; s < 2; ++s)
          p->nph_desc.push_back(NPhDesc{c.ext[v].off_NX[s], c.off_G, c.ext[v].off_GX, c.n, c.n + c.b, c.A,
                                        site_begin[i], s});
        B.dim(c.n + c.A);
      }
      B.end();
    }
    B.begin(S, ST_GEMM);  // N(contact rows) += Sigma^<_c conj(G(contact rows, Y))
    for (int i = 0; i < nc; ++i) {
      const Cluster& c = cl[i];
      const auto& x = c.ext[v];
      const int ldN = c.n + c.A, ldG = c.n + c.b;
      for (auto& ct : c.contacts) {
        const int m = p->contact_ptr[ct.first + 1] - p->contact_ptr[ct.first];
        const int64_t r0 = ct.second;
        for (int s = 0; s < 2; ++s) {
          const int64_t sig = AUX_BIT | (int64_t(s) * p->sigma_elems + soff[ct.first]);
          B.gemm(x.off_NX[s] + r0 * ldN, ldN, x.off_NX[s] + r0 * ldN, ldN, sig, m, OP_N, c.off_G + r0 * ldG, ldG, OP_C,
                 m, c.n, m, 1.0, 1.0);
          if (c.A)
            B.gemm(x.off_NX[s] + r0 * ldN + c.n, ldN, x.off_NX[s] + r0 * ldN + c.n, ldN, sig, m, OP_N,
                   x.off_GX + r0 * c.A, c.A, OP_C, m, c.A, m, 1.0, 1.0);
        }
      }
    }
    B.end();
    for (int l = 1; l <= p->n_levels; ++l) {  // fold N: N_{B,anc} += Psi^T N_{I,anc}, rows to the parent
      B.begin(S, ST_GEMM);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0 || !active(i)) continue;
        const auto& x = c.ext[v];
        for (int s = 0; s < 2; ++s)
          B.gemm(x.off_NB[s], c.A, x.off_NB[s], c.A, c.off_Psi, c.b, OP_T, x.off_NX[s] + c.n, c.n + c.A, OP_N, c.b,
                 c.A, c.n, 1.0, 1.0);
      }
      B.end();
      for (int sl = 0; sl <= max_slot; ++sl) {
        B.begin(S, ST_SCATTER_ROWS);
        for (int i : lev[l]) {
          const Cluster& c = cl[i];
          if (c.b == 0 || !active(i) || c.slot != sl) continue;
          const Cluster& P = cl[c.parent];
          for (int s = 0; s < 2; ++s)
            p->rows_desc.push_back(RowScatterDesc{c.ext[v].off_NB[s], P.ext[v].off_NX[s], P.ext[v].off_NB[s], c.b, c.A,
                                                  P.n, P.A, map_begin[i], P.k, site_begin[c.parent]});
          B.dim(c.b);
        }
        B.end();
      }
    }
    B.begin(S, ST_GEMM);  // P^(L-1) rows: A_ii^{-1} N_{I,Y}
    for (int i = 0; i < nc; ++i) {
      const Cluster& c = cl[i];
      if (!active(i)) continue;
      const int ldN = c.n + c.A;
      for (int s = 0; s < 2; ++s)
        B.gemm(c.ext[v].off_PX[s], ldN, c.ext[v].off_PX[s], ldN, c.off_F, c.n + c.b, OP_N, c.ext[v].off_NX[s], ldN,
               OP_N, c.n, ldN, c.n, 1.0, 0.0);
    }
    B.end();
    B.begin(S, ST_COLGATHER);  // [P_II | P_IB] = columns I_i, B_i of it
    for (int i = 0; i < nc; ++i) {
      const Cluster& c = cl[i];
      if (!active(i)) continue;
      for (int s = 0; s < 2; ++s)
        p->colg_desc.push_back(ColGatherDesc{c.off_P[s], c.ext[v].off_PX[s], c.n, c.b, c.A, cmap_begin[i],
                                             bsite_begin[i]});
      B.dim(c.n + c.b);
    }
    B.end();
    for (int l = p->n_levels; l >= 1; --l) {  // extract P
      B.begin(S, ST_GATHER_SKEW);
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0) continue;
        const Cluster& P = cl[c.parent];
        for (int s = 0; s < 2; ++s)
          p->gath_desc.push_back(GatherDesc{c.off_PBB[s], P.off_P[s], P.off_PBB[s], c.b, P.n, P.b, map_begin[i], P.k,
                                            site_begin[c.parent]});
        B.dim(c.b);
      }
      B.end();
      B.begin(S, ST_GEMM);  // P_IB = P_IB + Psi P_BB
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0) continue;
        const int ld = c.n + c.b;
        for (int s = 0; s < 2; ++s)
          B.gemm(c.off_P[s] + c.n, ld, c.off_P[s] + c.n, ld, c.off_Psi, c.b, OP_N, c.off_PBB[s], c.b, OP_N, c.n, c.b,
                 c.b, 1.0, active(i) ? 1.0 : 0.0);
      }
      B.end();
      B.begin(S, ST_GEMM);  // P_II = P_II + Psi P_BI,  P_BI = -(P_IB)^dagger
      for (int i : lev[l]) {
        const Cluster& c = cl[i];
        if (c.b == 0) continue;
        const int ld = c.n + c.b;
        for (int s = 0; s < 2; ++s)
          B.gemm(c.off_P[s], ld, c.off_P[s], ld, c.off_Psi, c.b, OP_N, c.off_P[s] + c.n, ld, OP_H, c.n, c.n, c.b,
                 -1.0, active(i) ? 1.0 : 0.0);
      }
      B.end();
    }
  }
  split_by_size(p, p->sched_factor);
  split_by_size(p, p->sched_green);
  split_by_size(p, p->sched_lesser[0]);
  split_by_size(p, p->sched_lesser[1]);
}

}  // namespace ndgf
