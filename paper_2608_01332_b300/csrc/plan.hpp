// Host-side contraction plan (Sec. X-A structural rounds; Alg. 1 step 1).
// Internal to libtlqr; the C ABI sees it as the opaque `tlqr_plan`.
#pragma once
#include <cstdint>
#include <vector>

struct tlqr_round {
  // Rakes of this round occupy [rake_begin, rake_end) of the rake arrays, grouped
  // by current parent (segments [seg_begin, seg_end)); leaves inside one segment
  // are in increasing node index (the sibling order of the reduction).
  int32_t rake_begin, rake_end;
  int32_t seg_begin, seg_end;
  // Compressions of this round occupy [comp_begin, comp_end), increasing centre index.
  int32_t comp_begin, comp_end;
};

struct tlqr_plan_t {
  int32_t N = 0;
  int32_t root = -1;                    // first root (the root of a single-tree plan)
  int32_t n_trees = 1;                  // roots in the parent array (a forest is a batch)
  std::vector<int32_t> parent;          // caller's parent array
  std::vector<tlqr_round> rounds;
  // rakes (global order: round by round, segment by segment)
  std::vector<int32_t> rake_leaf;       // j
  std::vector<int32_t> rake_parent;     // current parent i at rake time
  // absorb segments: contributions rake[seg_start[s] .. seg_start[s+1]) go to seg_parent[s]
  std::vector<int32_t> seg_parent;
  std::vector<int32_t> seg_start;       // size = #segments + 1
  // compressions
  std::vector<int32_t> comp_j, comp_i, comp_k;   // centre, current parent, current child
  // original-tree children (CSR), increasing index; for the KKT residual
  std::vector<int32_t> child_start, child_list;
  std::vector<int32_t> tree_of;         // forest: tree ordinal of each node (roots in increasing label)
  // per-node schedule (Fig. 2 labels)
  std::vector<int32_t> round_of_node, op_of_node;
  // statistics
  int32_t n_combine = 0, n_absorb = 0, levels = 0, height = 0, max_degree = 0;
};
