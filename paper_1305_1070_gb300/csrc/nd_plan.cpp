// S0 of the path: nested-dissection ordering, cluster tree, symbolic fold and
// the precomputed launch schedule (host only; runs without a GPU).
//
// Paper Sec. 3.2: each dissection step removes a small set of sites (the
// separator) that leaves two parts with no coupling between them, and is
// applied again to each part, which yields a binary cluster tree; clusters of
// one level never couple to each other and separators are kept small.
// Sec. 3.2, Fig. 8: the dense contact layers stay inside one cluster each.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <numeric>
#include <string>
#include <vector>

#include "nd_internal.h"

namespace ndgf {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

nd_status fail(nd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

namespace {

struct Node {
  std::vector<int> I;
  int parent = -1;
  std::vector<int> children;
};

// Recursive bisection with width-1 separators.
struct Dissector {
  int n = 0;
  std::vector<int> aptr, adj;  // adjacency without the diagonal
  int dim = 0;
  const double* coords = nullptr;
  std::vector<int> group;                   // contact id per site or -1
  std::vector<std::vector<int>> groups;     // sites of each contact
  std::vector<std::vector<double>> gcent;   // group centroid per axis
  int leaf = 64;
  int split = 500;  // cut position as a quantile of the keys, per mille
  int slab = 0;     // > 0: cuts along axis 0 leave slabs of this many distinct keys on the high side
  std::vector<Node> nodes;
  std::vector<int> mark;
  int tag = 0;

  int new_node(std::vector<int> I, int parent) {
    Node nd;
    nd.I = std::move(I);
    nd.parent = parent;
    nodes.push_back(std::move(nd));
    int id = int(nodes.size()) - 1;
    if (parent >= 0) nodes[parent].children.push_back(id);
    return id;
  }

  // Sort key of every site of D along the cut direction.  With coordinates:
  // the axis of largest extent over D (the first axis wins ties); otherwise
  // breadth-first distance from a pseudo-peripheral site.  A contact group
  // gets one key for all its sites so that a cut never splits it.
  int last_axis = -1;  // axis chosen by the last keys() call with coordinates
  void keys(const std::vector<int>& D, std::vector<double>& key) {
    key.assign(D.size(), 0.0);
    last_axis = -1;
    if (coords && dim > 0) {
      int best = 0;
      double bext = -1.0;
      for (int a = 0; a < dim; ++a) {
        double lo = 1e300, hi = -1e300;
        for (int v : D) {
          double x = coords[size_t(v) * dim + a];
          lo = std::min(lo, x);
          hi = std::max(hi, x);
        }
        if (hi - lo > bext * (1.0 + 1e-12) + 1e-12) {
          bext = hi - lo;
          best = a;
        }
      }
      for (size_t i = 0; i < D.size(); ++i) {
        int v = D[i];
        key[i] = group[v] >= 0 ? gcent[group[v]][best] : coords[size_t(v) * dim + best];
      }
      last_axis = best;
      return;
    }
    // breadth-first level structure inside D
    int inD = ++tag;
    for (int v : D) mark[v] = inD;
    std::vector<int> dist(n, -1);
    auto bfs = [&](int s, std::vector<int>& order) {
      for (int v : D) dist[v] = -1;
      order.clear();
      dist[s] = 0;
      order.push_back(s);
      for (size_t h = 0; h < order.size(); ++h) {
        int v = order[h];
        for (int p = aptr[v]; p < aptr[v + 1]; ++p) {
          int u = adj[p];
          if (mark[u] == inD && dist[u] < 0) {
            dist[u] = dist[v] + 1;
            order.push_back(u);
          }
        }
      }
    };
    std::vector<int> order;
    int s = D[0];
    for (int it = 0; it < 3; ++it) {
      bfs(s, order);
      s = order.back();
    }
    bfs(s, order);
    for (size_t i = 0; i < D.size(); ++i) {
      int v = D[i];
      key[i] = dist[v] < 0 ? 1e18 : double(dist[v]);
    }
    for (size_t i = 0; i < D.size(); ++i) {  // contact group: smallest key of its sites
      int g = group[D[i]];
      if (g < 0) continue;
      double kmin = key[i];
      for (size_t j = 0; j < D.size(); ++j)
        if (group[D[j]] == g) kmin = std::min(kmin, key[j]);
      key[i] = kmin;
    }
  }

  void leaf_node(std::vector<int>& D, int parent) { new_node(std::move(D), parent); }

  void rec(std::vector<int> D, int parent) {
    if (D.empty()) return;
    // groups inside D
    std::vector<int> gin;
    for (int v : D)
      if (group[v] >= 0 && std::find(gin.begin(), gin.end(), group[v]) == gin.end()) gin.push_back(group[v]);
    if (int(D.size()) <= leaf || (gin.size() == 1 && D.size() == groups[gin[0]].size())) {
      leaf_node(D, parent);
      return;
    }
    // a set that falls apart (several devices in one graph, or a cut that
    // isolated pieces) is dissected component by component under one parent
    {
      const int inD = ++tag;
      for (int v : D) mark[v] = inD;
      std::vector<std::vector<int>> comps;
      for (int v0 : D) {
        if (mark[v0] != inD) continue;
        const int seen = ++tag;
        std::vector<int> comp{v0};
        mark[v0] = seen;
        for (size_t h = 0; h < comp.size(); ++h)
          for (int p = aptr[comp[h]]; p < aptr[comp[h] + 1]; ++p)
            if (mark[adj[p]] == inD) {
              mark[adj[p]] = seen;
              comp.push_back(adj[p]);
            }
        comps.push_back(std::move(comp));
      }
      if (comps.size() > 1) {
        for (auto& comp : comps) {
          std::sort(comp.begin(), comp.end());
          rec(std::move(comp), parent);
        }
        return;
      }
    }
    std::vector<double> key;
    keys(D, key);
    std::vector<double> sk = key;
    std::sort(sk.begin(), sk.end());
    double c = sk[std::min(sk.size() - 1, size_t(double(sk.size()) * split / 1000.0))];
    if (slab > 0 && last_axis == 0) {
      // caterpillar cut: leave `slab` distinct key values (columns) above the
      // separator, so that the part below keeps the low-side contact
      std::vector<double> uk = sk;
      uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
      if (int(uk.size()) > slab + 1) c = uk[uk.size() - 1 - slab];
    }
    if (!(c > sk[0])) {
      auto it = std::upper_bound(sk.begin(), sk.end(), sk[0]);
      if (it == sk.end()) {  // cannot be split
        leaf_node(D, parent);
        return;
      }
      c = *it;
    }
    int tl = ++tag, tr = ++tag;
    std::vector<int> Lft, Rgt;
    for (size_t i = 0; i < D.size(); ++i) {
      if (key[i] < c) {
        mark[D[i]] = tl;
        Lft.push_back(D[i]);
      } else {
        mark[D[i]] = tr;
        Rgt.push_back(D[i]);
      }
    }
    std::vector<int> S, Rrest;
    for (int v : Rgt) {
      bool touches = false;
      for (int p = aptr[v]; p < aptr[v + 1] && !touches; ++p) touches = (mark[adj[p]] == tl);
      (touches ? S : Rrest).push_back(v);
    }
    // a contact group that the separator would cut is peeled off instead
    int bad = -1;
    for (int v : S)
      if (group[v] >= 0) {
        bad = group[v];
        break;
      }
    if (bad >= 0) {
      int inD = ++tag;
      for (int v : D) mark[v] = inD;
      int ing = ++tag;
      for (int v : groups[bad]) mark[v] = ing;
      int ins = ++tag;
      std::vector<int> Sg;
      for (int v : groups[bad])
        for (int p = aptr[v]; p < aptr[v + 1]; ++p) {
          int u = adj[p];
          if (mark[u] == inD) {
            mark[u] = ins;
            Sg.push_back(u);
          }
        }
      std::vector<int> rest;
      for (int v : D)
        if (mark[v] == inD) rest.push_back(v);
      std::vector<int> g = groups[bad];
      if (Sg.empty()) {
        new_node(std::move(g), parent);
        rec(std::move(rest), parent);
        return;
      }
      std::sort(Sg.begin(), Sg.end());
      int s = new_node(std::move(Sg), parent);
      new_node(std::move(g), s);
      rec(std::move(rest), s);
      return;
    }
    if (S.empty()) {  // the two sides are not connected inside D
      rec(std::move(Lft), parent);
      rec(std::move(Rrest), parent);
      return;
    }
    std::sort(S.begin(), S.end());
    int s = new_node(std::move(S), parent);
    rec(std::move(Lft), s);
    rec(std::move(Rrest), s);
  }
};

int64_t align16(int64_t x) { return (x + 15) & ~int64_t(15); }

}  // namespace

}  // namespace ndgf

using namespace ndgf;

extern "C" nd_status nd_analyze(const nd_graph* g, const nd_opts* opts, nd_plan** out) {
  if (!g || !out) return fail(ND_ERR_INVALID_ARG, "nd_analyze: NULL argument");
  *out = nullptr;
  const int n = g->n;
  if (n <= 0 || !g->rowptr || !g->colind) return fail(ND_ERR_INVALID_ARG, "nd_analyze: empty graph");
  if (g->rowptr[0] != 0) return fail(ND_ERR_INVALID_ARG, "nd_analyze: rowptr[0] != 0");
  for (int r = 0; r < n; ++r)
    if (g->rowptr[r + 1] < g->rowptr[r]) return fail(ND_ERR_INVALID_ARG, "nd_analyze: rowptr not monotone");
  const int nnz = g->rowptr[n];
  for (int p = 0; p < nnz; ++p)
    if (g->colind[p] < 0 || g->colind[p] >= n)
      return fail(ND_ERR_INVALID_ARG, "nd_analyze: column index out of range at " + std::to_string(p));
  if (g->n_contacts < 0 || (g->n_contacts > 0 && (!g->contact_ptr || !g->contact_idx)))
    return fail(ND_ERR_INVALID_ARG, "nd_analyze: bad contact arrays");
  if (g->coord_dim < 0 || (g->coord_dim > 0 && !g->coords))
    return fail(ND_ERR_INVALID_ARG, "nd_analyze: coord_dim > 0 needs coords");

  auto plan = new nd_plan();
  plan->n = n;
  plan->nnz = nnz;
  plan->rowptr.assign(g->rowptr, g->rowptr + n + 1);
  plan->colind.assign(g->colind, g->colind + nnz);

  Dissector d;
  d.n = n;
  d.leaf = (opts && opts->leaf_size > 0) ? opts->leaf_size : 64;
  d.split = (opts && opts->split_permille > 0) ? opts->split_permille : 500;
  d.slab = (opts && opts->slab > 0) ? opts->slab : 0;
  plan->delay = opts ? opts->delay : 0;
  if (plan->delay < 0 || plan->delay > 8) {
    delete plan;
    return fail(ND_ERR_INVALID_ARG, "nd_analyze: delay must be in 0..8");
  }
  if (d.split < 100 || d.split > 900) {
    delete plan;
    return fail(ND_ERR_INVALID_ARG, "nd_analyze: split_permille must be in 100..900");
  }
  d.dim = g->coord_dim;
  d.coords = g->coords;
  d.mark.assign(n, 0);
  // adjacency without the diagonal; structural symmetry check
  d.aptr.assign(n + 1, 0);
  for (int r = 0; r < n; ++r)
    for (int p = g->rowptr[r]; p < g->rowptr[r + 1]; ++p)
      if (g->colind[p] != r) d.aptr[r + 1]++;
  for (int r = 0; r < n; ++r) d.aptr[r + 1] += d.aptr[r];
  d.adj.resize(d.aptr[n]);
  {
    std::vector<int> fill(d.aptr.begin(), d.aptr.end() - 1);
    for (int r = 0; r < n; ++r)
      for (int p = g->rowptr[r]; p < g->rowptr[r + 1]; ++p)
        if (g->colind[p] != r) d.adj[fill[r]++] = g->colind[p];
    for (int r = 0; r < n; ++r) {
      std::sort(d.adj.begin() + d.aptr[r], d.adj.begin() + d.aptr[r + 1]);
      for (int p = d.aptr[r] + 1; p < d.aptr[r + 1]; ++p)
        if (d.adj[p] == d.adj[p - 1]) {
          delete plan;
          return fail(ND_ERR_INVALID_ARG, "nd_analyze: duplicate entry in row " + std::to_string(r));
        }
    }
    for (int r = 0; r < n; ++r)
      for (int p = d.aptr[r]; p < d.aptr[r + 1]; ++p) {
        int c = d.adj[p];
        if (!std::binary_search(d.adj.begin() + d.aptr[c], d.adj.begin() + d.aptr[c + 1], r)) {
          delete plan;
          return fail(ND_ERR_NOT_SYMMETRIC, "nd_analyze: pattern not symmetric at (" + std::to_string(r) +
                                                "," + std::to_string(c) + ")");
        }
      }
  }
  // contacts
  plan->n_contacts = g->n_contacts;
  d.group.assign(n, -1);
  if (g->n_contacts > 0) {
    plan->contact_ptr.assign(g->contact_ptr, g->contact_ptr + g->n_contacts + 1);
    int tot = plan->contact_ptr.back();
    if (plan->contact_ptr[0] != 0 || tot < 0) {
      delete plan;
      return fail(ND_ERR_INVALID_ARG, "nd_analyze: bad contact_ptr");
    }
    plan->contact_idx.assign(g->contact_idx, g->contact_idx + tot);
    d.groups.resize(g->n_contacts);
    for (int c = 0; c < g->n_contacts; ++c) {
      if (plan->contact_ptr[c + 1] <= plan->contact_ptr[c]) {
        delete plan;
        return fail(ND_ERR_INVALID_ARG, "nd_analyze: empty contact set");
      }
      for (int p = plan->contact_ptr[c]; p < plan->contact_ptr[c + 1]; ++p) {
        int v = plan->contact_idx[p];
        if (v < 0 || v >= n || d.group[v] >= 0) {
          delete plan;
          return fail(ND_ERR_INVALID_ARG, "nd_analyze: contact site out of range or in two contacts");
        }
        d.group[v] = c;
        d.groups[c].push_back(v);
      }
      plan->sigma_elems += int64_t(d.groups[c].size()) * int64_t(d.groups[c].size());
    }
    d.gcent.assign(g->n_contacts, std::vector<double>(std::max(1, d.dim), 0.0));
    if (d.coords)
      for (int c = 0; c < g->n_contacts; ++c)
        for (int a = 0; a < d.dim; ++a) {
          double s = 0;
          for (int v : d.groups[c]) s += d.coords[size_t(v) * d.dim + a];
          d.gcent[c][a] = s / double(d.groups[c].size());
        }
  }
  {
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    d.rec(std::move(all), -1);
  }
  // ---- postorder ------------------------------------------------------------
  const int nn = int(d.nodes.size());
  std::vector<int> post_of(nn, -1), order;
  order.reserve(nn);
  {
    std::vector<std::pair<int, int>> st;
    for (int r = 0; r < nn; ++r) {
      if (d.nodes[r].parent >= 0) continue;
      st.push_back({r, 0});
      while (!st.empty()) {
        auto& top = st.back();
        if (top.second < int(d.nodes[top.first].children.size())) {
          int c = d.nodes[top.first].children[top.second++];
          st.push_back({c, 0});
        } else {
          post_of[top.first] = int(order.size());
          order.push_back(top.first);
          st.pop_back();
        }
      }
    }
  }
  auto& cl = plan->cl;
  cl.resize(nn);
  for (int i = 0; i < nn; ++i) {
    const Node& nd = d.nodes[order[i]];
    Cluster& c = cl[i];
    c.parent = nd.parent >= 0 ? post_of[nd.parent] : -1;
    for (int ch : nd.children) c.children.push_back(post_of[ch]);
    std::sort(c.children.begin(), c.children.end());
    c.I = nd.I;
  }
  plan->owner.assign(n, -1);
  plan->pos.assign(n, -1);
  for (int i = 0; i < nn; ++i) {
    Cluster& c = cl[i];
    // contact sites first, in contact order
    std::vector<int> cids;
    for (int v : c.I)
      if (d.group[v] >= 0 && std::find(cids.begin(), cids.end(), d.group[v]) == cids.end()) cids.push_back(d.group[v]);
    std::sort(cids.begin(), cids.end());
    std::vector<int> I;
    for (int cid : cids) {
      c.contacts.push_back({cid, int(I.size())});
      for (int v : d.groups[cid]) I.push_back(v);
    }
    std::vector<int> rest;
    for (int v : c.I)
      if (d.group[v] < 0) rest.push_back(v);
    std::sort(rest.begin(), rest.end());
    I.insert(I.end(), rest.begin(), rest.end());
    if (I.size() != c.I.size()) {
      delete plan;
      return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (contact split across clusters)");
    }
    c.I = I;
    c.n = int(I.size());
    c.n_own = c.n;
    for (int k = 0; k < c.n; ++k) {
      plan->owner[I[k]] = i;
      plan->pos[I[k]] = k;
    }
    c.slot = 0;
    c.first_desc = i;
    c.level = 1;
    for (int ch : c.children) {
      c.first_desc = std::min(c.first_desc, cl[ch].first_desc);
      c.level = std::max(c.level, cl[ch].level + 1);
    }
    for (size_t s = 0; s < c.children.size(); ++s) cl[c.children[s]].slot = int(s);
    c.nactive = !c.contacts.empty();
    for (int ch : c.children) c.nactive = c.nactive || cl[ch].nactive;
  }
  for (int v = 0; v < n; ++v)
    if (plan->owner[v] < 0) {
      delete plan;
      return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (site not in a cluster)");
    }
  // ---- symbolic fold: boundary sets B_i --------------------------------------
  {
    std::vector<int> seen(n, -1);
    for (int i = 0; i < nn; ++i) {
      Cluster& c = cl[i];
      std::vector<int> B;
      auto consider = [&](int u) -> bool {
        int o = plan->owner[u];
        if (o == i || (o >= c.first_desc && o < i)) return true;  // inside the subtree
        if (o < c.first_desc || cl[o].first_desc > i) return false; // not an ancestor
        if (seen[u] != i) {
          seen[u] = i;
          B.push_back(u);
        }
        return true;
      };
      for (int v : c.I)
        for (int p = d.aptr[v]; p < d.aptr[v + 1]; ++p)
          if (!consider(d.adj[p])) {
            delete plan;
            return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (clusters of one level couple)");
          }
      for (int ch : c.children)
        for (int u : cl[ch].B)
          if (!consider(u)) {
            delete plan;
            return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (boundary not in ancestors)");
          }
      std::sort(B.begin(), B.end(), [&](int a, int b2) {
        if (plan->owner[a] != plan->owner[b2]) return plan->owner[a] < plan->owner[b2];
        return plan->pos[a] < plan->pos[b2];
      });
      c.B = B;
      c.b = int(B.size());
      if (c.parent < 0 && c.b != 0) {
        delete plan;
        return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (root with boundary)");
      }
    }
    // Delayed pivots: in postorder (children first), every eligible cluster
    // hands k of its front rows to its parent as virtual unknowns (ids n, n+1,
    // ...), appended to the parent's front rows and put first in its own
    // boundary.  They couple only to the cluster's boundary, which lies in
    // the parent's front, so the boundary sets above stay valid.
    if (plan->delay > 0) {
      int nv = 0;
      for (int i = 0; i < nn; ++i) {
        Cluster& c = cl[i];
        const int nfr = int(c.I.size());
        const int k = (c.parent >= 0 && c.contacts.empty() && c.b > 0 && nfr >= 2) ? std::min(plan->delay, nfr - 1) : 0;
        c.k = k;
        c.n = nfr - k;
        if (k == 0) continue;
        Cluster& P = cl[c.parent];
        c.dslot = int(P.I.size());
        std::vector<int> Bn;
        for (int j = 0; j < k; ++j) {
          const int v = n + nv++;
          plan->owner.push_back(c.parent);
          plan->pos.push_back(int(P.I.size()));
          P.I.push_back(v);
          Bn.push_back(v);
        }
        Bn.insert(Bn.end(), c.B.begin(), c.B.end());
        c.B = std::move(Bn);
        c.b = int(c.B.size());
      }
      plan->n_virtual = nv;
    }
    // maps into the parent's front: front rows [0, n_p + k_p) in their static
    // order, then the parent's boundary entries (positions n_p + index in B_p)
    std::vector<int> posB(n + plan->n_virtual, -1);
    for (int p = 0; p < nn; ++p) {
      Cluster& P = cl[p];
      for (int k = 0; k < P.b; ++k) posB[P.B[k]] = k;
      for (int ch : P.children) {
        Cluster& c = cl[ch];
        c.map.resize(c.b);
        for (int k = 0; k < c.b; ++k) {
          int u = c.B[k];
          int m;
          if (plan->owner[u] == p) {
            m = plan->pos[u];
          } else if (posB[u] >= P.k && P.B[posB[u]] == u) {
            m = P.n + posB[u];
          } else {
            delete plan;
            return fail(ND_ERR_INVALID_ARG, "nd_analyze: internal error (child boundary outside parent front)");
          }
          c.map[k] = m;
        }
      }
      for (int k = 0; k < P.b; ++k) posB[P.B[k]] = -1;
    }
  }
  // ---- levels, sizes, workspace layout, flop model --------------------------
  for (int i = nn - 1; i >= 0; --i) {  // parents come after children in postorder
    Cluster& c = cl[i];
    c.A = c.parent >= 0 ? cl[c.parent].A + cl[c.parent].n : 0;
  }
  int64_t off = 0;
  double ff = 0, fg = 0, fl = 0;
  for (int i = 0; i < nn; ++i) {
    Cluster& c = cl[i];
    const int64_t nI = c.n, b = c.b, F = nI * (nI + b), Ff = int64_t(c.nf()) * (nI + b);
    plan->n_levels = std::max(plan->n_levels, c.level);
    plan->max_n = std::max(plan->max_n, c.nf());
    plan->max_b = std::max(plan->max_b, c.b);
    if (c.parent < 0) plan->n_roots++;
    c.off_F = off; off = align16(off + Ff);
    c.off_Psi = off; off = align16(off + nI * b);
    c.off_BB = off; off = align16(off + b * b);
    c.off_G = off; off = align16(off + Ff);
    for (int s = 0; s < 2; ++s) {
      c.off_PBB[s] = off; off = align16(off + b * b);
      c.off_P[s] = off; off = align16(off + F);
    }
    const double dn = double(nI), db = double(b), dA = double(c.A);
    ff += 8.0 * (dn * dn * dn + dn * dn * db + dn * db * db);
    fg += 8.0 * (dn * db * db + dn * dn * db);
    double lesser = 2.0 * (dn * db * db + dn * dn * db);  // P extraction, both sides
    if (c.nactive) lesser += dn * db * dA + 2.0 * (db * dn * dA + dn * dn * (dn + dA));  // G_{I,anc}, N fold, P^(L-1)
    for (auto& ct : c.contacts) {
      double m = double(plan->contact_ptr[ct.first + 1] - plan->contact_ptr[ct.first]);
      lesser += 2.0 * m * m * (dn + dA);  // N = Sigma^< conj(G)
    }
    fl += 8.0 * lesser;
  }
  // G^< blocks over ancestor columns: variant 0 = clusters whose subtree holds
  // a contact, variant 1 = every cluster (a phonon self-energy on all sites)
  for (int v = 0; v < 2; ++v) {
    int64_t eo = off;
    for (int i = 0; i < nn; ++i) {
      Cluster& c = cl[i];
      if (v == 0 && !c.nactive) continue;
      const int64_t nI = c.n, b = c.b, A = c.A, W = nI * (nI + A);
      auto& x = c.ext[v];
      x.off_GX = eo; eo = align16(eo + nI * A);
      x.off_GBA = eo; eo = align16(eo + b * A);
      for (int s = 0; s < 2; ++s) {
        x.off_NX[s] = eo; eo = align16(eo + W);
        x.off_NB[s] = eo; eo = align16(eo + b * A);
        x.off_PX[s] = eo; eo = align16(eo + W);
      }
    }
    plan->ext_elems[v] = eo - off;
  }
  plan->arena_elems = off;
  // adjoint blocks (used only by workspaces created with ND_FACT_ADJOINT)
  {
    const int64_t M = plan->n_contacts > 0 ? plan->contact_ptr[plan->n_contacts] : 0;
    plan->adj_cols = int32_t(M);
    int64_t ao = 0;
    for (auto& c : cl) {
      const int64_t m = c.n, b = c.b;
      c.adj_XI = ao; ao = align16(ao + m * M);
      c.adj_RB = ao; ao = align16(ao + b * M);
      c.adj_XB = ao; ao = align16(ao + b * M);
      c.adj_XS = ao; ao = align16(ao + m * M);
      c.adj_U = ao; ao = align16(ao + m * M);
    }
    plan->adj_elems = ao;
  }
  plan->flops_factor = ff;
  plan->flops_green_r = fg;
  plan->flops_green_lesser = fl;
  try {
    build_schedules(plan);
  } catch (const std::exception& ex) {
    delete plan;
    return fail(ND_ERR_INVALID_ARG, std::string("nd_analyze: internal error building the schedule: ") + ex.what());
  }
  *out = plan;
  return ND_OK;
}

extern "C" nd_status nd_plan_query(const nd_plan* p, nd_plan_info* out) {
  if (!p || !out) return fail(ND_ERR_INVALID_ARG, "nd_plan_query: NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->n = p->n;
  out->nnz = p->nnz;
  out->n_clusters = int32_t(p->cl.size());
  out->n_levels = p->n_levels;
  out->max_n = p->max_n;
  out->max_b = p->max_b;
  out->n_contacts = p->n_contacts;
  out->n_roots = p->n_roots;
  out->flops_factor = p->flops_factor;
  out->flops_green_r = p->flops_green_r;
  out->flops_green_lesser = p->flops_green_lesser;
  out->arena_bytes_fp64 = double(p->arena_elems + p->ext_elems[0]) * 16.0;
  out->arena_bytes_fp32 = double(p->arena_elems + p->ext_elems[0]) * 8.0;
  return ND_OK;
}

extern "C" nd_status nd_plan_tree(const nd_plan* p, int32_t* level, int32_t* parent, int32_t* n_i,
                                  int32_t* b_i, int32_t* cluster_of_site) {
  if (!p) return fail(ND_ERR_INVALID_ARG, "nd_plan_tree: NULL plan");
  for (size_t i = 0; i < p->cl.size(); ++i) {
    if (level) level[i] = p->cl[i].level;
    if (parent) parent[i] = p->cl[i].parent;
    if (n_i) n_i[i] = p->cl[i].nf();
    if (b_i) b_i[i] = p->cl[i].b;
  }
  if (cluster_of_site)
    for (int v = 0; v < p->n; ++v) cluster_of_site[v] = p->owner[v];
  return ND_OK;
}

extern "C" nd_status nd_plan_cluster_sites(const nd_plan* p, int32_t c, int32_t* sites) {
  if (!p || !sites) return fail(ND_ERR_INVALID_ARG, "nd_plan_cluster_sites: NULL argument");
  if (c < 0 || c >= int32_t(p->cl.size())) return fail(ND_ERR_INVALID_ARG, "nd_plan_cluster_sites: bad cluster");
  const Cluster& C = p->cl[c];
  std::copy(C.I.begin(), C.I.end(), sites);
  std::copy(C.B.begin(), C.B.end(), sites + C.nf());
  return ND_OK;
}

extern "C" void nd_plan_destroy(nd_plan* p) { delete p; }

extern "C" const char* nd_last_error(void) { return ndgf::g_err.c_str(); }

extern "C" const char* nd_version(void) { return "ndgf 0.1 (sm_103a)"; }
