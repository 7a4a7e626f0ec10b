// Host planner: parent[] -> structural rake/compress rounds (Sec. X-A).
//
// Each round rakes every nonroot leaf of the current tree and then compresses a
// maximal set of pairwise nonadjacent unary nonroot nodes, chosen greedily in
// increasing node index: a unary node is taken unless its current parent or
// current child was already taken in this round.  The paper's planner scans all
// node slots per round (O(N log N), Sec. X-C remark); this one keeps a list of
// live nodes, so a round costs O(live nodes) and the whole plan O(N) because
// every round removes at least a third of them (Lemma 2).
//
// The plan also records the dependency levels of eq. (earliest-level), with
// sibling contributions combined by the readiness-weighted alphabetic
// reduction of eq. (readiness-code-data) (Lemma 3).  The GPU executor runs
// round by round and sums siblings in the same (increasing index) order; the
// levels are reported for comparison with Tab. I and the bound of Lemma 4.
#include <algorithm>
#include <new>

#include "../../include/tlqr.h"
#include "plan.hpp"

namespace {

using u128 = unsigned __int128;

// Readiness-weighted reduction of eq. (readiness-code-data): weights 2^l_j,
// codewords = first d_j^0 bits of the Shannon-Fano-Elias midpoints, binary trie
// with unary vertices contracted.  Returns the level of the final aggregate and
// adds the number of combinations to *n_comb; returns -1 if the weights do not
// fit the exact 128-bit arithmetic used here.
struct Code { u128 r; int len; int level; };

int trie_level(std::vector<Code>& codes, int lo, int hi, int pos, int* n_comb) {
  if (hi - lo == 1) return codes[lo].level;
  // codes are sorted (order preserving); find the first with bit `pos` = 1
  int mid = lo;
  while (mid < hi && ((codes[mid].r >> (codes[mid].len - 1 - pos)) & 1) == 0) ++mid;
  if (mid == lo || mid == hi) return trie_level(codes, lo, hi, pos + 1, n_comb);
  ++*n_comb;
  int a = trie_level(codes, lo, mid, pos + 1, n_comb);
  int b = trie_level(codes, mid, hi, pos + 1, n_comb);
  return 1 + std::max(a, b);
}

int readiness_level(const std::vector<int>& lv, int* n_comb) {
  const int k = (int)lv.size();
  if (k == 1) return lv[0];
  int lmin = *std::min_element(lv.begin(), lv.end());
  int lmax = *std::max_element(lv.begin(), lv.end());
  // normalised weights 2^(l - lmin); W < 2^(spread + 1 + log2 k) must stay < 2^60
  int logk = 0;
  while ((1 << logk) < k) ++logk;
  if (lmax - lmin + logk + 1 > 60) return -1;
  std::vector<u128> w(k);
  u128 W = 0;
  for (int j = 0; j < k; ++j) { w[j] = (u128)1 << (lv[j] - lmin); W += w[j]; }
  std::vector<Code> codes(k);
  u128 S = 0;
  for (int j = 0; j < k; ++j) {
    int d = 0;                                  // ceil(log2(W / w_j))
    while ((w[j] << d) < W) ++d;
    int d0 = d + 1;
    // first d0 bits of m_j = (2 S + w_j) / (2 W)
    u128 num = (2 * S + w[j]) << d0;
    codes[j] = Code{num / (2 * W), d0, lv[j]};
    S += w[j];
  }
  return trie_level(codes, 0, k, 0, n_comb);
}

}  // namespace

namespace {

// Shared builder.  allow_forest = false: exactly one root; true: one or more
// roots, each tree contracted independently in the same rounds (a batch).
int build_plan(const int32_t* parent, int32_t N, bool allow_forest, tlqr_plan_t** out) {
  if (!parent || !out || N < 1) return TLQR_ERR_ARG;
  *out = nullptr;
  tlqr_plan_t* P = new (std::nothrow) tlqr_plan_t;
  if (!P) return TLQR_ERR_OOM;
  try {
    P->N = N;
    P->parent.assign(parent, parent + N);
    int root = -1, n_roots = 0;
    for (int i = 0; i < N; ++i) {
      int p = parent[i];
      if (p == -1) {
        if (root >= 0 && !allow_forest) { delete P; return TLQR_ERR_TOPOLOGY; }
        if (root < 0) root = i;
        ++n_roots;
      } else if (p < 0 || p >= N || p == i) {
        delete P;
        return TLQR_ERR_TOPOLOGY;
      }
    }
    if (root < 0) { delete P; return TLQR_ERR_TOPOLOGY; }
    P->root = root;
    P->n_trees = n_roots;

    // original children, CSR in increasing index
    std::vector<int32_t> cnt(N, 0);
    P->child_start.assign(N + 1, 0);
    for (int j = 0; j < N; ++j) if (parent[j] >= 0) P->child_start[parent[j] + 1]++;
    for (int i = 0; i < N; ++i) P->child_start[i + 1] += P->child_start[i];
    P->child_list.resize(std::max(0, N - 1));
    {
      std::vector<int32_t> fill(P->child_start.begin(), P->child_start.end() - 1);
      for (int j = 0; j < N; ++j) if (parent[j] >= 0) P->child_list[fill[parent[j]]++] = j;
    }
    // reachability from the root (a cycle leaves nodes unreached) and height
    {
      std::vector<int32_t> depth(N, -1), stack;
      P->tree_of.assign(N, 0);
      for (int i = 0, t = 0; i < N; ++i)
        if (parent[i] < 0) { depth[i] = 0; P->tree_of[i] = t++; stack.push_back(i); }
      int seen = 0;
      while (!stack.empty()) {
        int i = stack.back(); stack.pop_back(); ++seen;
        int deg = P->child_start[i + 1] - P->child_start[i];
        P->max_degree = std::max(P->max_degree, deg);
        for (int t = P->child_start[i]; t < P->child_start[i + 1]; ++t) {
          int j = P->child_list[t];
          depth[j] = depth[i] + 1;
          P->tree_of[j] = P->tree_of[i];
          P->height = std::max(P->height, depth[j]);
          stack.push_back(j);
        }
      }
      if (seen != N) { delete P; return TLQR_ERR_TOPOLOGY; }
    }

    // current tree state
    std::vector<int32_t> cur_parent(parent, parent + N);
    std::vector<int32_t> nchild(N, 0);
    std::vector<int64_t> child_sum(N, 0);       // sum of current child ids (gives the only child)
    for (int j = 0; j < N; ++j) if (parent[j] >= 0) { nchild[parent[j]]++; child_sum[parent[j]] += j; }
    std::vector<char> selected(N, 0), dead(N, 0);
    std::vector<int32_t> live;
    live.reserve(N);
    for (int i = 0; i < N; ++i) live.push_back(i);
    P->round_of_node.assign(N, 0);
    P->op_of_node.assign(N, TLQR_OP_ROOT);

    // dependency levels (eq. earliest-level)
    std::vector<int32_t> lvU(N, 0), lvE(N, 0);
    int max_level = 0;
    bool level_overflow = false;

    std::vector<int32_t> leaves, sel;
    int round_no = 0;
    while ((int)live.size() > n_roots) {
      ++round_no;
      tlqr_round rd{};
      // ---- rake every nonroot leaf
      leaves.clear();
      for (int32_t j : live) if (parent[j] >= 0 && nchild[j] == 0) leaves.push_back(j);
      // group by current parent, keeping increasing leaf index inside a group
      std::stable_sort(leaves.begin(), leaves.end(),
                       [&](int a, int b) { return cur_parent[a] < cur_parent[b]; });
      rd.rake_begin = (int32_t)P->rake_leaf.size();
      rd.seg_begin = (int32_t)P->seg_parent.size();
      std::vector<int> seg_levels;
      for (size_t t = 0; t < leaves.size(); ++t) {
        int j = leaves[t], i = cur_parent[j];
        if (t == 0 || cur_parent[leaves[t - 1]] != i) {
          P->seg_parent.push_back(i);
          P->seg_start.push_back((int32_t)P->rake_leaf.size());
        }
        P->rake_leaf.push_back(j);
        P->rake_parent.push_back(i);
        P->round_of_node[j] = round_no;
        P->op_of_node[j] = TLQR_OP_RAKE;
      }
      rd.rake_end = (int32_t)P->rake_leaf.size();
      rd.seg_end = (int32_t)P->seg_parent.size();
      // levels of rakes, reductions, absorptions
      for (int s = rd.seg_begin; s < rd.seg_end; ++s) {
        int b = P->seg_start[s];
        int e = (s + 1 < rd.seg_end) ? P->seg_start[s + 1] : rd.rake_end;
        int i = P->seg_parent[s];
        seg_levels.clear();
        for (int t = b; t < e; ++t) {
          int j = P->rake_leaf[t];
          int lv = 1 + std::max(lvU[j], lvE[j]);
          seg_levels.push_back(lv);
          max_level = std::max(max_level, lv);
        }
        int agg = readiness_level(seg_levels, &P->n_combine);
        if (agg < 0) { level_overflow = true; agg = *std::max_element(seg_levels.begin(), seg_levels.end()) + 64; }
        lvU[i] = 1 + std::max(lvU[i], agg);
        max_level = std::max({max_level, agg, lvU[i]});
        P->n_absorb++;
      }
      for (int32_t j : leaves) {
        int i = cur_parent[j];
        nchild[i]--;
        child_sum[i] -= j;
        dead[j] = 1;
      }
      // ---- greedy nonadjacent compressions in increasing index
      rd.comp_begin = (int32_t)P->comp_j.size();
      sel.clear();
      for (int32_t j : live) {
        if (dead[j] || parent[j] < 0 || nchild[j] != 1) continue;
        int k = (int)child_sum[j];
        int i = cur_parent[j];
        if (selected[i] || selected[k]) continue;
        selected[j] = 1;
        sel.push_back(j);
        P->comp_j.push_back(j);
        P->comp_i.push_back(i);
        P->comp_k.push_back(k);
        P->round_of_node[j] = round_no;
        P->op_of_node[j] = TLQR_OP_COMPRESS;
      }
      rd.comp_end = (int32_t)P->comp_j.size();
      for (int t = rd.comp_begin; t < rd.comp_end; ++t) {
        int j = P->comp_j[t], i = P->comp_i[t], k = P->comp_k[t];
        int lv = 1 + std::max({lvU[j], lvE[j], lvE[k]});
        lvE[k] = lv;
        max_level = std::max(max_level, lv);
        child_sum[i] += (int64_t)k - j;
        cur_parent[k] = i;
        dead[j] = 1;
      }
      for (int32_t j : sel) selected[j] = 0;
      if (rd.rake_end == rd.rake_begin && rd.comp_end == rd.comp_begin) {
        delete P;
        return TLQR_ERR_TOPOLOGY;  // cannot happen for a tree
      }
      P->rounds.push_back(rd);
      // compact the live list
      size_t w = 0;
      for (size_t t = 0; t < live.size(); ++t) if (!dead[live[t]]) live[w++] = live[t];
      live.resize(w);
    }
    P->seg_start.push_back((int32_t)P->rake_leaf.size());
    P->levels = level_overflow ? -1 : max_level;
  } catch (const std::bad_alloc&) {
    delete P;
    return TLQR_ERR_OOM;
  }
  *out = P;
  return TLQR_OK;
}

}  // namespace

extern "C" int tlqr_plan_create(const int32_t* parent, int32_t N, tlqr_plan_t** out) {
  return build_plan(parent, N, false, out);
}

extern "C" int tlqr_plan_create_forest(const int32_t* parent, int32_t N, tlqr_plan_t** out) {
  return build_plan(parent, N, true, out);
}

extern "C" void tlqr_plan_destroy(tlqr_plan_t* plan) { delete plan; }

extern "C" int tlqr_plan_stats(const tlqr_plan_t* P, tlqr_plan_stats_t* out) {
  if (!P || !out) return TLQR_ERR_ARG;
  out->N = P->N;
  out->root = P->root;
  out->rounds = (int32_t)P->rounds.size();
  out->n_rake = (int32_t)P->rake_leaf.size();
  out->n_compress = (int32_t)P->comp_j.size();
  out->n_combine = P->n_combine;
  out->n_absorb = P->n_absorb;
  out->levels = P->levels;
  out->height = P->height;
  out->max_degree = P->max_degree;
  out->n_trees = P->n_trees;
  return TLQR_OK;
}

extern "C" int tlqr_plan_schedule(const tlqr_plan_t* P, int32_t* round_of_node, int32_t* op_of_node) {
  if (!P) return TLQR_ERR_ARG;
  if (round_of_node) std::copy(P->round_of_node.begin(), P->round_of_node.end(), round_of_node);
  if (op_of_node) std::copy(P->op_of_node.begin(), P->op_of_node.end(), op_of_node);
  return TLQR_OK;
}
