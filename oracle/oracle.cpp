// Oracle: a plain, slow, single-threaded CPU statement of the deterministic
// coarsening step and the deterministic lambda-1 label-propagation pass of
// Mt-KaHyPar (arXiv 2303.17679).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: only the tests, the smoke check and the benchmark's CPU
// baseline do.  It shares no code, header, table or helper with the CUDA
// library; the two meet only in the seeded inputs they are both given.
//
// Every routine follows a definition or a rule of the paper, cited by section
// and equation.  Data structures are the obvious ones (std::vector, std::map,
// std::set); there is no blocking, fusion or reordering beyond what the rule
// itself states, so each function can be checked against the paper by eye.
//
// Readings of points the paper leaves open (all integer, so results are
// bit-exact):
//  * sub-round of a node: mix64(seed ^ level<<32 ^ u) mod S for clustering,
//    mix64(seed ^ level<<32 ^ (pass+1)<<48 ^ u) mod S for label propagation,
//    mix64 = the SplitMix64 output function (Steele, Lea, Flood 2014);
//  * heavy-edge rating in Q20 fixed point, each net term floored:
//    floor(w(e) * 2^20 / (|e| - 1)); a net counts once per distinct cluster;
//    nets with |e| > T are skipped; ties go to the smaller cluster id;
//  * a candidate cluster C is skipped if it is u itself, if it is an
//    unclustered node of the same sub-round, or if cw[C] + c(u) > c_max;
//  * c_max = ceil(W / (f * k)) with W the total node weight and f = 160;
//  * clustering stops before a sub-round once 5 * clusters <= 2 * n;
//  * a level is not built when n <= f * k; after a level, coarsening ends when
//    100 * n' > 99 * n (the level is kept);
//  * identical nets: representative = smallest net id, weights summed,
//    coarse nets ordered by representative id, pins ascending;
//  * L_max = floor(ceil(W / k) * (10^6 + eps_ppm) / 10^6);
//  * label-propagation pair selection: per-pair slack
//    floor(max(0, L_max - c(V_i)) / (k - 1)); walk the merge path of the two
//    weight-prefix sequences (step into M_st while A[i] <= B[j]) and keep the
//    last feasible state;
//  * initial partition: nodes in order of (mix64(seed ^ 2^63 ^ u), u), each to
//    the currently lightest block, ties to the smaller block id;
//  * community detection (Sec. 4 "Community-Aware Coarsening", Sec. 11
//    "Deterministic Louvain Method"): the bipartite graph of the hypergraph
//    (a vertex per node, a vertex n + e per net, an edge {v, n + e} per pin)
//    with edge weight floor(w(e) * 2^20 / |e|), an integer reading of the
//    fractional w(e) / |e| model; modularity moves compared exactly in 128-bit
//    integers; vertices in sub-rounds mix64(seed ^ 2^62 ^ level<<32 ^
//    (round+1)<<48 ^ i) mod S; up to 5 rounds per Louvain level, ending after
//    a round that moved fewer than 1 % of the vertices; a Louvain level
//    without any move ends the detection (as do 32 levels); a candidate
//    cluster of the coarsening rating must lie in u's community.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC oracle.cpp -o liboracle.so
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <stdexcept>
#include <tuple>
#include <utility>
#include <vector>

namespace {

using std::vector;

// ------------------------------------------------------------------ hashing

// SplitMix64 output function applied to the state x (first output of a
// SplitMix64 generator seeded with x).
uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int subround_clustering(uint64_t seed, int level, int u, int S) {
  uint64_t key = seed ^ ((uint64_t)(uint32_t)level << 32) ^ (uint64_t)(uint32_t)u;
  return (int)(mix64(key) % (uint64_t)S);
}

int subround_lp(uint64_t seed, int level, int pass, int u, int S) {
  uint64_t key = seed ^ ((uint64_t)(uint32_t)level << 32) ^ ((uint64_t)(uint32_t)(pass + 1) << 48) ^
                 (uint64_t)(uint32_t)u;
  return (int)(mix64(key) % (uint64_t)S);
}

uint64_t initial_key(uint64_t seed, int u) {
  return mix64(seed ^ (1ULL << 63) ^ (uint64_t)(uint32_t)u);
}

// ------------------------------------------------------------- hypergraph

// H = (V, E, c, w) as in Sec. 2 "Hypergraphs": pin lists of the nets and,
// derived from them, the incident nets I(u) of every node.
struct Hypergraph {
  int n = 0, m = 0;
  vector<vector<int>> pins;  // pins[e]
  vector<int> w;             // w(e)
  vector<int> c;             // c(u)
  vector<vector<int>> inc;   // I(u), ascending net ids
};

Hypergraph load(int n, int m, const int32_t* off, const int32_t* pins, const int32_t* w,
                const int32_t* c) {
  Hypergraph h;
  h.n = n;
  h.m = m;
  h.pins.resize(m);
  h.w.resize(m);
  h.c.resize(n);
  h.inc.resize(n);
  for (int e = 0; e < m; ++e) {
    h.w[e] = w ? w[e] : 1;
    for (int q = off[e]; q < off[e + 1]; ++q) {
      h.pins[e].push_back(pins[q]);
      h.inc[pins[q]].push_back(e);
    }
  }
  for (int u = 0; u < n; ++u) h.c[u] = c ? c[u] : 1;
  return h;
}

int64_t total_weight(const Hypergraph& h) {
  int64_t W = 0;
  for (int u = 0; u < h.n; ++u) W += h.c[u];
  return W;
}

// ------------------------------------------------------- partition values

// Phi(e, V_i) = |e ∩ V_i| (Sec. 2, "Clusterings and Partitions").
vector<vector<int>> pin_counts(const Hypergraph& h, int k, const int32_t* part) {
  vector<vector<int>> phi(h.m, vector<int>(k, 0));
  for (int e = 0; e < h.m; ++e)
    for (int v : h.pins[e]) phi[e][part[v]] += 1;
  return phi;
}

// lambda(e) = |Lambda(e)|, Lambda(e) = blocks with Phi(e, V_i) > 0.
int connectivity(const vector<int>& phi_e) {
  int l = 0;
  for (int x : phi_e) l += (x > 0);
  return l;
}

// Connectivity objective f_{lambda-1} = sum over cut nets of (lambda(e) - 1) w(e)
// (Sec. 2, "The Balanced Hypergraph Partitioning Problem").
int64_t objective_from_phi(const Hypergraph& h, const vector<vector<int>>& phi) {
  int64_t f = 0;
  for (int e = 0; e < h.m; ++e) {
    int l = connectivity(phi[e]);
    if (l > 1) f += (int64_t)(l - 1) * h.w[e];
  }
  return f;
}

// Gain of moving u to V_t (Sec. 6, definition of g_u(V_t)):
// w({e in I(u) : Phi(e, Pi[u]) = 1}) - w({e in I(u) : Phi(e, V_t) = 0}).
int64_t gain(const Hypergraph& h, const vector<vector<int>>& phi, const int32_t* part, int u,
             int t) {
  int64_t benefit = 0, penalty = 0;
  for (int e : h.inc[u]) {
    if (phi[e][part[u]] == 1) benefit += h.w[e];
    if (phi[e][t] == 0) penalty += h.w[e];
  }
  return benefit - penalty;
}

// L_max = (1 + eps) * ceil(c(V) / k) (Sec. 2), eps given in parts per million.
int64_t balance_limit(int64_t W, int k, int eps_ppm) {
  int64_t per_block = (W + k - 1) / k;
  return per_block * (1000000 + (int64_t)eps_ppm) / 1000000;
}

// ----------------------------------------------------- label propagation

struct Move {
  int u, from, to;
  int64_t g;
};

struct LPState {
  const Hypergraph* h;
  int k;
  int64_t lmax;
  vector<int32_t> part;
  vector<vector<int>> phi;
  vector<int64_t> bw;  // c(V_i)
};

// One synchronous sub-round of deterministic label propagation (Sec. 11,
// "Deterministic Label Propagation Refinement"):
//  1. every node of the sub-round computes its best move from the current
//     (snapshot) state, kept only if its gain is positive;
//  2. for every block pair the two move sequences are sorted by (gain desc,
//     id asc) and the last feasible prefix pair on the merge path is chosen;
//  3. the chosen moves are applied (Algorithm 3's pin-count updates, without
//     the concurrency).
// Returns the candidate moves and, aligned with them, which were applied.
std::pair<vector<Move>, vector<char>> lp_subround(LPState& st, uint64_t seed, int level, int pass,
                                                  int s, int S) {
  const Hypergraph& h = *st.h;
  const int k = st.k;
  vector<Move> moves;
  for (int u = 0; u < h.n; ++u) {
    if (subround_lp(seed, level, pass, u, S) != s) continue;
    const int from = st.part[u];
    int best_t = -1;
    int64_t best_g = 0;  // only strictly positive gains qualify
    for (int t = 0; t < k; ++t) {
      if (t == from) continue;
      int64_t g = gain(h, st.phi, st.part.data(), u, t);
      if (g > best_g) {  // strict: ties keep the smaller block id
        best_g = g;
        best_t = t;
      }
    }
    if (best_t >= 0) moves.push_back({u, from, best_t, best_g});
  }

  vector<char> applied(moves.size(), 0);
  auto by_gain_then_id = [&](int a, int b) {
    if (moves[a].g != moves[b].g) return moves[a].g > moves[b].g;
    return moves[a].u < moves[b].u;
  };
  for (int a = 0; a < k; ++a) {
    for (int b = a + 1; b < k; ++b) {
      vector<int> Mab, Mba;  // indices into moves
      for (int i = 0; i < (int)moves.size(); ++i) {
        if (moves[i].from == a && moves[i].to == b) Mab.push_back(i);
        if (moves[i].from == b && moves[i].to == a) Mba.push_back(i);
      }
      if (Mab.empty() && Mba.empty()) continue;
      std::sort(Mab.begin(), Mab.end(), by_gain_then_id);
      std::sort(Mba.begin(), Mba.end(), by_gain_then_id);
      // A[i] = weight of the first i moves a->b, B[j] likewise for b->a
      vector<int64_t> A(Mab.size() + 1, 0), B(Mba.size() + 1, 0);
      for (size_t i = 0; i < Mab.size(); ++i) A[i + 1] = A[i] + h.c[moves[Mab[i]].u];
      for (size_t j = 0; j < Mba.size(); ++j) B[j + 1] = B[j] + h.c[moves[Mba[j]].u];
      const int64_t slack_a = std::max<int64_t>(0, st.lmax - st.bw[a]) / (k - 1);
      const int64_t slack_b = std::max<int64_t>(0, st.lmax - st.bw[b]) / (k - 1);
      // x(i, j) = A[i] - B[j] is the weight that block b gains and block a loses.
      auto feasible = [&](size_t i, size_t j) {
        int64_t x = A[i] - B[j];
        return -slack_a <= x && x <= slack_b;
      };
      size_t i = 0, j = 0, bi = 0, bj = 0;  // (0, 0) is always feasible
      while (i < Mab.size() || j < Mba.size()) {
        // advance the sequence whose source block currently receives more
        // weight: x <= 0 means block a is not lighter, so move a->b next
        if (i < Mab.size() && (j == Mba.size() || A[i] <= B[j])) ++i;
        else ++j;
        if (feasible(i, j)) { bi = i; bj = j; }
      }
      for (size_t q = 0; q < bi; ++q) applied[Mab[q]] = 1;
      for (size_t q = 0; q < bj; ++q) applied[Mba[q]] = 1;
    }
  }

  for (size_t i = 0; i < moves.size(); ++i) {
    if (!applied[i]) continue;
    const Move& mv = moves[i];
    st.part[mv.u] = mv.to;
    st.bw[mv.from] -= h.c[mv.u];
    st.bw[mv.to] += h.c[mv.u];
    for (int e : h.inc[mv.u]) {
      st.phi[e][mv.from] -= 1;
      st.phi[e][mv.to] += 1;
    }
  }
  return {moves, applied};
}

// --------------------------------------------------------------- clustering

struct Contraction {
  Hypergraph coarse;
  vector<int> map;  // fine node -> coarse node
};

// Contraction of a clustering given by representatives (Sec. 4.2): every
// cluster becomes one node whose weight is the sum of its members' weights
// (coarse ids by rank of the representative); every pin is replaced by its
// cluster, repeated pins are discarded, single-pin nets are removed, and
// identical nets are merged into the one with the smallest id, whose weight
// becomes the sum of the group.  Coarse nets are listed in order of their
// representative's id, pins ascending.
Contraction contract(const Hypergraph& h, const vector<int>& rep) {
  Contraction out;
  const int n = h.n;
  vector<int> cid(n, -1);
  int n2 = 0;
  for (int u = 0; u < n; ++u)
    if (rep[u] == u) cid[u] = n2++;
  Hypergraph& H2 = out.coarse;
  H2.n = n2;
  H2.c.assign(n2, 0);
  out.map.resize(n);
  for (int u = 0; u < n; ++u) {
    if (cid[rep[u]] < 0) throw std::logic_error("rep[u] is not a representative");
    out.map[u] = cid[rep[u]];
    H2.c[out.map[u]] += h.c[u];
  }
  std::map<vector<int>, std::pair<int, int64_t>> identical;  // pin set -> (first net, weight)
  for (int e = 0; e < h.m; ++e) {
    vector<int> s;
    for (int v : h.pins[e]) s.push_back(out.map[v]);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    if (s.size() < 2) continue;
    auto it = identical.find(s);
    if (it == identical.end()) identical.emplace(s, std::make_pair(e, (int64_t)h.w[e]));
    else it->second.second += h.w[e];
  }
  vector<std::tuple<int, const vector<int>*, int64_t>> order;
  for (auto& kv : identical) order.emplace_back(kv.second.first, &kv.first, kv.second.second);
  std::sort(order.begin(), order.end(),
            [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
  H2.m = (int)order.size();
  H2.inc.assign(n2, {});
  for (int e2 = 0; e2 < H2.m; ++e2) {
    H2.pins.push_back(*std::get<1>(order[e2]));
    H2.w.push_back((int)std::get<2>(order[e2]));
    for (int v : H2.pins.back()) H2.inc[v].push_back(e2);
  }
  return out;
}

struct CoarsenResult {
  bool stop_before = false;  // no level built (n <= f * k)
  bool stop_after = false;   // level built, but it shrank by less than 1 %
  vector<int> rep, target, rated_in;
  Hypergraph coarse;
  vector<int> map;  // fine node -> coarse node
};

// One deterministic clustering level followed by contraction (Sec. 4.1 rating
// function, contraction limit and c_max; Sec. 11 "Deterministic Clustering for
// Coarsening"; Sec. 4.2 contraction and identical-net removal).
CoarsenResult coarsen(const Hypergraph& h, int64_t W, int k, int S, int T, int factor, uint64_t seed,
                      int level, const vector<int>* comm = nullptr) {
  CoarsenResult res;
  const int n = h.n;
  if ((int64_t)n <= (int64_t)factor * k) {
    res.stop_before = true;
    return res;
  }
  const int64_t c_max = (W + (int64_t)factor * k - 1) / ((int64_t)factor * k);

  vector<int> rep(n);
  vector<int64_t> cw(n);
  vector<char> joined(n, 0);  // false while u is a singleton cluster (unclustered)
  vector<int> target(n, -2), rated_in(n, -1);
  for (int u = 0; u < n; ++u) {
    rep[u] = u;
    cw[u] = h.c[u];
  }
  int64_t clusters = n;

  for (int s = 0; s < S; ++s) {
    if (5 * clusters <= 2 * (int64_t)n) break;
    // --- targets from the state at the start of the sub-round
    vector<std::pair<int, int>> moves;  // (u, C)
    for (int u = 0; u < n; ++u) {
      if (joined[u] || subround_clustering(seed, level, u, S) != s) continue;
      rated_in[u] = s;
      std::map<int, int64_t> rating;  // r(u, C) for every admissible C
      for (int e : h.inc[u]) {
        const int size = (int)h.pins[e].size();
        if (size < 2 || size > T) continue;
        const int64_t term = ((int64_t)h.w[e] << 20) / (size - 1);
        std::set<int> clusters_of_e;
        for (int v : h.pins[e]) clusters_of_e.insert(rep[v]);
        for (int C : clusters_of_e) {
          if (C == u) continue;
          // community-aware coarsening (Sec. 4): contractions stay inside a
          // community (every member of C shares C's community)
          if (comm && (*comm)[C] != (*comm)[u]) continue;
          if (!joined[C] && subround_clustering(seed, level, C, S) == s) continue;
          if (cw[C] + h.c[u] > c_max) continue;
          rating[C] += term;
        }
      }
      int best = -1;
      int64_t best_r = -1;
      for (const auto& kv : rating) {  // ascending C, strict > keeps the smaller id
        if (kv.second > best_r) {
          best_r = kv.second;
          best = kv.first;
        }
      }
      target[u] = best;
      if (best >= 0) moves.push_back({u, best});
    }
    // --- approval: per target, (c(u) asc, id asc), longest prefix within c_max
    std::map<int, vector<int>> groups;
    for (auto& mv : moves) groups[mv.second].push_back(mv.first);
    for (auto& g : groups) {
      const int C = g.first;
      vector<int>& members = g.second;
      if (rep[C] != C) throw std::logic_error("target is not a representative");
      std::sort(members.begin(), members.end(), [&](int a, int b) {
        if (h.c[a] != h.c[b]) return h.c[a] < h.c[b];
        return a < b;
      });
      int64_t added = 0;
      int accepted = 0;
      for (int u : members) {
        if (cw[C] + added + h.c[u] > c_max) break;
        added += h.c[u];
        ++accepted;
      }
      for (int q = 0; q < accepted; ++q) {
        rep[members[q]] = C;
        joined[members[q]] = 1;
      }
      if (accepted > 0) {
        joined[C] = 1;
        cw[C] += added;
        clusters -= accepted;
      }
    }
  }

  Contraction con = contract(h, rep);
  res.coarse = std::move(con.coarse);
  res.map = std::move(con.map);
  const int n2 = res.coarse.n;
  res.rep = rep;
  res.target = target;
  res.rated_in = rated_in;
  res.stop_after = 100 * (int64_t)n2 > 99 * (int64_t)n;
  return res;
}

// ------------------------------------------------------------ communities

// A weighted undirected graph for the Louvain method: adjacency lists (no
// self entries) and a self-loop weight per vertex.  The degree of vertex i is
// k_i = sum_j A_ij + 2 self_i, and 2W = sum_i k_i.
struct LGraph {
  int V = 0;
  vector<vector<std::pair<int, int64_t>>> adj;  // (neighbour, weight)
  vector<int64_t> self;
};

int64_t lg_degree(const LGraph& g, int i) {
  int64_t k = 2 * g.self[i];
  for (auto& a : g.adj[i]) k += a.second;
  return k;
}

// The bipartite graph of a hypergraph (Sec. 4, "Community-Aware Coarsening"):
// vertex v for node v, vertex n + e for net e, an edge {v, n + e} for every
// pin v of e with weight floor(w(e) * 2^20 / |e|).
LGraph bipartite_graph(const Hypergraph& h) {
  LGraph g;
  g.V = h.n + h.m;
  g.adj.assign(g.V, {});
  g.self.assign(g.V, 0);
  for (int e = 0; e < h.m; ++e) {
    const int64_t we = ((int64_t)h.w[e] << 20) / (int64_t)h.pins[e].size();
    for (int v : h.pins[e]) {
      g.adj[v].push_back({h.n + e, we});
      g.adj[h.n + e].push_back({v, we});
    }
  }
  return g;
}

int subround_louvain(uint64_t seed, int level, int round, int i, int S) {
  uint64_t key = seed ^ (1ULL << 62) ^ ((uint64_t)(uint32_t)level << 32) ^
                 ((uint64_t)(uint32_t)(round + 1) << 48) ^ (uint64_t)(uint32_t)i;
  return (int)(mix64(key) % (uint64_t)S);
}

// The best cluster for vertex i given the clustering cl and the cluster
// volumes vol (Sec. 11, synchronous local moving): moving i from its cluster
// A into C changes the modularity by (2 / (2W)^2) (s(C) - s(A)) with
// s(C) = 2W k_{i,C} - k_i vol(C) for C != A and
// s(A) = 2W k_{i,A} - k_i (vol(A) - k_i), k_{i,C} the weight of i's edges
// into C.  Candidates are the clusters of i's neighbours; the largest s wins,
// ties to the smaller cluster id; i moves only if s(best) > s(A).  Returns
// the target, or -1 to stay.
int louvain_best_move(const LGraph& g, const vector<int>& cl, const vector<int64_t>& vol,
                      int64_t W2, int i) {
  const int A = cl[i];
  const int64_t ki = lg_degree(g, i);
  std::map<int, int64_t> kic;  // k_{i,C} of every neighbouring cluster
  for (auto& a : g.adj[i]) kic[cl[a.first]] += a.second;
  using i128 = __int128;
  const int64_t kia = kic.count(A) ? kic[A] : 0;
  const i128 s_own = (i128)W2 * kia - (i128)ki * (vol[A] - ki);
  int best = -1;
  i128 best_s = 0;
  for (auto& kv : kic) {  // ascending C: strict > keeps the smaller id on ties
    if (kv.first == A) continue;
    const i128 sc = (i128)W2 * kv.second - (i128)ki * vol[kv.first];
    if (best < 0 || sc > best_s) {
      best = kv.first;
      best_s = sc;
    }
  }
  if (best >= 0 && best_s > s_own) return best;
  return -1;
}

// Aggregation (the Louvain method's coarsening of the graph): clusters become
// vertices numbered by the rank of their cluster id; edges between clusters
// are summed, edges inside a cluster add to its self-loop weight.
LGraph louvain_aggregate(const LGraph& g, const vector<int>& cl, vector<int>& cid) {
  cid.assign(g.V, -1);
  vector<char> used(g.V, 0);
  for (int i = 0; i < g.V; ++i) used[cl[i]] = 1;
  int V2 = 0;
  for (int c = 0; c < g.V; ++c)
    if (used[c]) cid[c] = V2++;
  LGraph h;
  h.V = V2;
  h.adj.assign(V2, {});
  h.self.assign(V2, 0);
  vector<std::map<int, int64_t>> acc(V2);
  vector<int64_t> internal(V2, 0);  // inside a cluster, each edge seen from both ends
  for (int i = 0; i < g.V; ++i) {
    const int ci = cid[cl[i]];
    h.self[ci] += g.self[i];
    for (auto& a : g.adj[i]) {
      const int cj = cid[cl[a.first]];
      if (cj == ci) internal[ci] += a.second;
      else acc[ci][cj] += a.second;
    }
  }
  for (int c = 0; c < V2; ++c) {
    h.self[c] += internal[c] / 2;
    for (auto& kv : acc[c]) h.adj[c].push_back(kv);
  }
  return h;
}

struct LouvainStats {
  int levels = 0;
  int64_t moves = 0;
};

// Deterministic Louvain method on the bipartite graph (Sec. 4, Sec. 11):
// per level, up to max_rounds rounds of S synchronous sub-rounds (every
// vertex of a sub-round picks its move from the state at the sub-round's
// start; all moves are applied, cluster volumes updated by integer sums), a
// round moving fewer than 1 % of the vertices ends the level; then the
// clusters are aggregated into the next level's vertices.  Returns the
// community of every hypergraph node, numbered by the rank of the final
// cluster ids.
vector<int> communities(const Hypergraph& h, int S, uint64_t seed, int max_rounds, int max_levels,
                        LouvainStats& st) {
  LGraph g = bipartite_graph(h);
  vector<int> vmap(h.n);  // hypergraph node -> vertex of the current level
  for (int v = 0; v < h.n; ++v) vmap[v] = v;
  int64_t W2 = 0;
  for (int i = 0; i < g.V; ++i) W2 += lg_degree(g, i);
  vector<int> cl;
  for (int level = 0; level < max_levels; ++level) {
    cl.assign(g.V, 0);
    vector<int64_t> vol(g.V);
    for (int i = 0; i < g.V; ++i) {
      cl[i] = i;
      vol[i] = lg_degree(g, i);
    }
    int64_t level_moves = 0;
    for (int round = 0; round < max_rounds; ++round) {
      int64_t moved = 0;
      for (int s = 0; s < S; ++s) {
        vector<std::pair<int, int>> moves;
        for (int i = 0; i < g.V; ++i) {
          if (subround_louvain(seed, level, round, i, S) != s) continue;
          const int t = louvain_best_move(g, cl, vol, W2, i);
          if (t >= 0) moves.push_back({i, t});
        }
        for (auto& mv : moves) {
          const int64_t ki = lg_degree(g, mv.first);
          vol[cl[mv.first]] -= ki;
          vol[mv.second] += ki;
          cl[mv.first] = mv.second;
        }
        moved += (int64_t)moves.size();
      }
      level_moves += moved;
      if (100 * moved < (int64_t)g.V) break;
    }
    st.moves += level_moves;
    if (level_moves == 0) break;
    st.levels = level + 1;
    vector<int> cid;
    LGraph next = louvain_aggregate(g, cl, cid);
    for (int v = 0; v < h.n; ++v) vmap[v] = cid[cl[vmap[v]]];
    const bool shrank = next.V < g.V;
    g = std::move(next);
    cl.clear();
    if (!shrank) break;
  }
  // every level either ended without a move or was aggregated, so the
  // communities are the vertices of the last graph (numbered 0..V-1 by rank)
  return vmap;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

uint64_t o_mix64(uint64_t x) { return mix64(x); }

int32_t o_subround_clustering(uint64_t seed, int32_t level, int32_t u, int32_t S) {
  return subround_clustering(seed, level, u, S);
}

int32_t o_subround_lp(uint64_t seed, int32_t level, int32_t pass, int32_t u, int32_t S) {
  return subround_lp(seed, level, pass, u, S);
}

// Phi as a dense m x k int32 table and Lambda as one 64-bit mask per net (k <= 64).
void o_pin_counts(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, int32_t k,
                  const int32_t* part, int32_t* phi, uint64_t* lambda) {
  Hypergraph h = load(n, m, off, pins, nullptr, nullptr);
  auto p = pin_counts(h, k, part);
  for (int e = 0; e < m; ++e) {
    uint64_t mask = 0;
    for (int i = 0; i < k; ++i) {
      phi[(int64_t)e * k + i] = p[e][i];
      if (p[e][i] > 0) mask |= 1ULL << i;
    }
    if (lambda) lambda[e] = mask;
  }
}

int64_t o_objective(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                    const int32_t* w, int32_t k, const int32_t* part) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  return objective_from_phi(h, pin_counts(h, k, part));
}

// Gains g_u(V_t) of all nodes to all blocks (t == Pi[u] gives 0 by definition
// of "no move"): out is n x k int64.
void o_gains(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, const int32_t* w,
             int32_t k, const int32_t* part, int64_t* out) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  auto phi = pin_counts(h, k, part);
  for (int u = 0; u < n; ++u)
    for (int t = 0; t < k; ++t)
      out[(int64_t)u * k + t] = (t == part[u]) ? 0 : gain(h, phi, part, u, t);
}

// Exact gains of a move sequence M = <m_1, ..., m_l>, m_i = (u_i, Pi[u_i],
// t_i), each node moved at most once (Sec. 6.3, "The Parallel Gain
// Recalculation Algorithm"): g_i is the gain of Sec. 6 of moving u_i to t_i
// in the partition reached after m_1 .. m_{i-1}, i.e. the objective decrease
// that m_i causes when the moves are performed in this order.  Evaluated here
// by performing the moves one by one on the pin counts.  Returns 0, or 1 for
// a node moved twice, a target outside [0, k) or equal to the node's block.
int32_t o_recalculate_gains(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                            const int32_t* w, int32_t k, const int32_t* part, int32_t l,
                            const int32_t* nodes, const int32_t* targets, int64_t* gains) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  vector<int32_t> cur(part, part + n);
  vector<char> moved(n, 0);
  for (int i = 0; i < l; ++i) {
    const int u = nodes[i], t = targets[i];
    if (u < 0 || u >= n || moved[u] || t < 0 || t >= k || t == part[u]) return 1;
    moved[u] = 1;
  }
  auto phi = pin_counts(h, k, cur.data());
  for (int i = 0; i < l; ++i) {
    const int u = nodes[i], t = targets[i], s = cur[u];
    gains[i] = gain(h, phi, cur.data(), u, t);
    for (int e : h.inc[u]) {
      phi[e][s] -= 1;
      phi[e][t] += 1;
    }
    cur[u] = t;
  }
  return 0;
}

// Gain table (Sec. 6.2): benefit b(u) = w({e in I(u) : Phi(e, Pi[u]) = 1})
// and penalty p(u, V_i) = w({e in I(u) : Phi(e, V_i) = 0}) for every block,
// from their definitions; b is n int64, p is n x k int64.
void o_gain_table(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, const int32_t* w,
                  int32_t k, const int32_t* part, int64_t* b, int64_t* p) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  auto phi = pin_counts(h, k, part);
  for (int u = 0; u < n; ++u) {
    int64_t bu = 0;
    for (int e : h.inc[u])
      if (phi[e][part[u]] == 1) bu += h.w[e];
    b[u] = bu;
    for (int i = 0; i < k; ++i) {
      int64_t pu = 0;
      for (int e : h.inc[u])
        if (phi[e][i] == 0) pu += h.w[e];
      p[(int64_t)u * k + i] = pu;
    }
  }
}

void o_block_weights(int32_t n, const int32_t* c, int32_t k, const int32_t* part, int64_t* bw) {
  for (int i = 0; i < k; ++i) bw[i] = 0;
  for (int u = 0; u < n; ++u) bw[part[u]] += c ? c[u] : 1;
}

int64_t o_balance_limit(int64_t W, int32_t k, int32_t eps_ppm) { return balance_limit(W, k, eps_ppm); }

// Label propagation refinement: up to max_passes passes of S sub-rounds each;
// a pass that applies no move ends the refinement.  part is updated in place.
// Optional outputs: phi_out (m x k, maintained incrementally), per-(pass,
// sub-round) counts of candidate and applied moves (max_passes * S each).
// Returns 0, or -1 for invalid arguments.
int32_t o_lp_refine(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                    const int32_t* w, const int32_t* c, int32_t k, int32_t eps_ppm, int32_t S,
                    uint64_t seed, int32_t level, int32_t max_passes, int32_t* part,
                    int64_t* out_objective, int64_t* out_moves, int32_t* out_passes,
                    int32_t* phi_out, int64_t* trace_candidates, int64_t* trace_applied) {
  if (k < 2 || k > 64 || S < 1 || max_passes < 0) return -1;
  Hypergraph h = load(n, m, off, pins, w, c);
  LPState st;
  st.h = &h;
  st.k = k;
  st.lmax = balance_limit(total_weight(h), k, eps_ppm);
  st.part.assign(part, part + n);
  st.phi = pin_counts(h, k, part);
  st.bw.assign(k, 0);
  for (int u = 0; u < n; ++u) st.bw[st.part[u]] += h.c[u];
  int64_t total_moves = 0;
  int passes = 0;
  for (int pass = 0; pass < max_passes; ++pass) {
    ++passes;
    int64_t moved = 0;
    for (int s = 0; s < S; ++s) {
      auto r = lp_subround(st, seed, level, pass, s, S);
      int64_t a = 0;
      for (char x : r.second) a += x;
      moved += a;
      if (trace_candidates) trace_candidates[(int64_t)pass * S + s] = (int64_t)r.first.size();
      if (trace_applied) trace_applied[(int64_t)pass * S + s] = a;
    }
    total_moves += moved;
    if (moved == 0) break;
  }
  std::copy(st.part.begin(), st.part.end(), part);
  if (out_objective) *out_objective = objective_from_phi(h, st.phi);
  if (out_moves) *out_moves = total_moves;
  if (out_passes) *out_passes = passes;
  if (phi_out)
    for (int e = 0; e < m; ++e)
      for (int i = 0; i < k; ++i) phi_out[(int64_t)e * k + i] = st.phi[e][i];
  return 0;
}

// One label-propagation sub-round from the given partition (Phi and block
// weights rebuilt from part).  Writes the candidate moves (u, from, to, gain,
// applied) into the five output arrays (capacity n) and returns their number.
int32_t o_lp_subround(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                      const int32_t* w, const int32_t* c, int32_t k, int32_t eps_ppm, int32_t S,
                      uint64_t seed, int32_t level, int32_t pass, int32_t s, int32_t* part,
                      int32_t* mv_u, int32_t* mv_from, int32_t* mv_to, int64_t* mv_gain,
                      int8_t* mv_applied) {
  if (k < 2 || k > 64) return -1;
  Hypergraph h = load(n, m, off, pins, w, c);
  LPState st;
  st.h = &h;
  st.k = k;
  st.lmax = balance_limit(total_weight(h), k, eps_ppm);
  st.part.assign(part, part + n);
  st.phi = pin_counts(h, k, part);
  st.bw.assign(k, 0);
  for (int u = 0; u < n; ++u) st.bw[st.part[u]] += h.c[u];
  auto r = lp_subround(st, seed, level, pass, s, S);
  for (size_t i = 0; i < r.first.size(); ++i) {
    mv_u[i] = r.first[i].u;
    mv_from[i] = r.first[i].from;
    mv_to[i] = r.first[i].to;
    mv_gain[i] = r.first[i].g;
    mv_applied[i] = r.second[i];
  }
  std::copy(st.part.begin(), st.part.end(), part);
  return (int32_t)r.first.size();
}

// One clustering + contraction level.  Return: 1 = no level (n <= factor*k),
// 0 = level built.  Outputs (capacities: n for node arrays, m+1 / p / m for the
// coarse net CSR): rep, target (-2 not rated, -1 no candidate), rated_in
// (sub-round, -1 if never rated), map (fine -> coarse), the coarse hypergraph
// in canonical order, and *stop_after = 1 if the level shrank by < 1 %.
// comm (n entries, may be NULL): community of every node; candidates outside
// u's community are skipped, and ccomm (capacity n) receives the coarse
// nodes' communities.
int32_t o_coarsen(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                  const int32_t* w, const int32_t* c, int64_t W, int32_t k, int32_t S, int32_t T,
                  int32_t factor, uint64_t seed, int32_t level, int32_t* rep, int32_t* target,
                  int32_t* rated_in, int32_t* map, int32_t* out_n, int32_t* out_m, int64_t* out_p,
                  int32_t* coff, int32_t* cpins, int32_t* cw, int32_t* cc, int32_t* stop_after,
                  const int32_t* comm, int32_t* ccomm) {
  Hypergraph h = load(n, m, off, pins, w, c);
  vector<int> cm;
  if (comm) cm.assign(comm, comm + n);
  CoarsenResult r = coarsen(h, W, k, S, T, factor, seed, level, comm ? &cm : nullptr);
  if (r.stop_before) return 1;
  // coarse communities: every cluster lies inside one community
  if (comm && ccomm)
    for (int u = 0; u < n; ++u) ccomm[r.map[u]] = cm[u];
  std::copy(r.rep.begin(), r.rep.end(), rep);
  std::copy(r.target.begin(), r.target.end(), target);
  std::copy(r.rated_in.begin(), r.rated_in.end(), rated_in);
  std::copy(r.map.begin(), r.map.end(), map);
  const Hypergraph& H2 = r.coarse;
  *out_n = H2.n;
  *out_m = H2.m;
  int64_t p = 0;
  coff[0] = 0;
  for (int e = 0; e < H2.m; ++e) {
    for (int v : H2.pins[e]) cpins[p++] = v;
    coff[e + 1] = (int32_t)p;
    cw[e] = H2.w[e];
  }
  *out_p = p;
  for (int v = 0; v < H2.n; ++v) cc[v] = H2.c[v];
  *stop_after = r.stop_after ? 1 : 0;
  return 0;
}

// Contraction of an arbitrary clustering (rep[u] = representative of u's
// cluster, rep[rep[u]] == rep[u]).  Output capacities as for o_coarsen.
// Returns 0, or -1 if rep is not a valid representative array.
int32_t o_contract(int32_t n, int32_t m, const int32_t* off, const int32_t* pins,
                   const int32_t* w, const int32_t* c, const int32_t* rep, int32_t* map,
                   int32_t* out_n, int32_t* out_m, int64_t* out_p, int32_t* coff, int32_t* cpins,
                   int32_t* cw, int32_t* cc) {
  Hypergraph h = load(n, m, off, pins, w, c);
  vector<int> r(rep, rep + n);
  for (int u = 0; u < n; ++u)
    if (r[u] < 0 || r[u] >= n || r[r[u]] != r[u]) return -1;
  Contraction con = contract(h, r);
  std::copy(con.map.begin(), con.map.end(), map);
  const Hypergraph& H2 = con.coarse;
  *out_n = H2.n;
  *out_m = H2.m;
  int64_t p = 0;
  coff[0] = 0;
  for (int e = 0; e < H2.m; ++e) {
    for (int v : H2.pins[e]) cpins[p++] = v;
    coff[e + 1] = (int32_t)p;
    cw[e] = H2.w[e];
  }
  *out_p = p;
  for (int v = 0; v < H2.n; ++v) cc[v] = H2.c[v];
  return 0;
}

// Bipartite graph of a hypergraph (Sec. 4): V = n + m vertices, CSR
// adjacency (capacity 2p) with weights floor(w(e) * 2^20 / |e|).
void o_bipartite(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, const int32_t* w,
                 int64_t* boff, int32_t* badj, int64_t* bw) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  LGraph g = bipartite_graph(h);
  int64_t q = 0;
  boff[0] = 0;
  for (int i = 0; i < g.V; ++i) {
    for (auto& a : g.adj[i]) {
      badj[q] = a.first;
      bw[q] = a.second;
      ++q;
    }
    boff[i + 1] = q;
  }
}

namespace {
LGraph lgraph_from(int32_t V, const int64_t* off, const int32_t* adj, const int64_t* w,
                   const int64_t* self) {
  LGraph g;
  g.V = V;
  g.adj.assign(V, {});
  g.self.assign(V, 0);
  for (int i = 0; i < V; ++i) {
    g.self[i] = self ? self[i] : 0;
    for (int64_t q = off[i]; q < off[i + 1]; ++q) g.adj[i].push_back({adj[q], w[q]});
  }
  return g;
}
}  // namespace

// One Louvain move decision (see louvain_best_move) for vertex i of a graph
// in CSR form with self-loop weights, clustering cl and volumes vol.
int32_t o_louvain_best_move(int32_t V, const int64_t* off, const int32_t* adj, const int64_t* w,
                            const int64_t* self, const int32_t* cl, const int64_t* vol, int32_t i) {
  LGraph g = lgraph_from(V, off, adj, w, self);
  vector<int> c(cl, cl + V);
  vector<int64_t> vo(vol, vol + V);
  int64_t W2 = 0;
  for (int x = 0; x < V; ++x) W2 += lg_degree(g, x);
  return louvain_best_move(g, c, vo, W2, i);
}

// Aggregation of a clustering (see louvain_aggregate).  Outputs: V2, the
// coarse CSR (capacity: V + 1 offsets, the input's entries), self-loop
// weights and cid (cluster id -> coarse vertex, -1 for unused ids).
void o_louvain_aggregate(int32_t V, const int64_t* off, const int32_t* adj, const int64_t* w,
                         const int64_t* self, const int32_t* cl, int32_t* out_V2, int64_t* off2,
                         int32_t* adj2, int64_t* w2, int64_t* self2, int32_t* cid_out) {
  LGraph g = lgraph_from(V, off, adj, w, self);
  vector<int> c(cl, cl + V), cid;
  LGraph h = louvain_aggregate(g, c, cid);
  *out_V2 = h.V;
  int64_t q = 0;
  off2[0] = 0;
  for (int i = 0; i < h.V; ++i) {
    for (auto& a : h.adj[i]) {
      adj2[q] = a.first;
      w2[q] = a.second;
      ++q;
    }
    off2[i + 1] = q;
    self2[i] = h.self[i];
  }
  for (int x = 0; x < V; ++x) cid_out[x] = cid[x];
}

// Communities of the hypergraph's nodes (Sec. 4, Sec. 11; see communities).
// stats: [0] Louvain levels aggregated, [1] vertex moves.
void o_communities(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, const int32_t* w,
                   int32_t S, uint64_t seed, int32_t max_rounds, int32_t max_levels, int32_t* comm,
                   int64_t* stats) {
  Hypergraph h = load(n, m, off, pins, w, nullptr);
  LouvainStats st;
  vector<int> c = communities(h, S, seed, max_rounds, max_levels, st);
  std::copy(c.begin(), c.end(), comm);
  if (stats) {
    stats[0] = st.levels;
    stats[1] = st.moves;
  }
}

// Projection Pi_fine[u] = Pi_coarse[map[u]] (Algorithm 1, uncoarsening).
void o_project(int32_t n_fine, const int32_t* map, const int32_t* coarse_part, int32_t* fine_part) {
  for (int u = 0; u < n_fine; ++u) fine_part[u] = coarse_part[map[u]];
}

// Seeded balanced initial partition (a stand-in for the paper's portfolio,
// Sec. 5): nodes in order of (mix64(seed ^ 2^63 ^ u), u); each goes to the
// lightest block so far, ties to the smaller block id.
void o_initial_partition(int32_t n, const int32_t* c, int32_t k, uint64_t seed, int32_t* part) {
  vector<std::pair<uint64_t, int>> order(n);
  for (int u = 0; u < n; ++u) order[u] = {initial_key(seed, u), u};
  std::sort(order.begin(), order.end());
  vector<int64_t> bw(k, 0);
  for (auto& kv : order) {
    int u = kv.second, best = 0;
    for (int b = 1; b < k; ++b)
      if (bw[b] < bw[best]) best = b;
    part[u] = best;
    bw[best] += c ? c[u] : 1;
  }
}

}  // extern "C"
