// Non-overlapping domain decomposition of the spacetree along its depth-first
// cell order (paper Sec. 3, distributed memory: the cells are split into
// contiguous ranges of the space-filling-curve order; Riemann problems on
// faces between two partitions are solved on both sides, and the predictor
// results of the cells along a partition boundary are sent to the neighbour
// once per step; those cells join the skeleton so that their predictions run
// first and the enclave predictions hide the exchange).
//
// Cuts fall on base-cell boundaries: every family of 3^d siblings then lies in
// one partition, so refinement and coarsening move no data across partitions
// and a remesh only shifts whole base-cell subtrees between neighbours in the
// order when the cuts are rebalanced.
#pragma once
#include <cstdint>
#include <vector>

#include "mesh.h"

namespace ader {

struct SubDomain {
  int nranks = 1, rank = 0;
  std::vector<int64_t> base_cut;   // nranks + 1 cuts in base-cell indices (x fastest)
  std::vector<int64_t> cut;        // the same cuts as tree cell indices
  int64_t first = 0;               // owned cells: tree cells [first, first + lists.nowned)
  std::vector<int32_t> ghosts;     // tree index of ghost g = local cell nowned + g (ascending)
  MeshLists lists;                 // in local numbering
  // Face data exchanged each step, per peer rank: entries local_cell * 2d +
  // slot (slot = 2 dir + side), both sides ordered by (tree cell, slot).
  std::vector<std::vector<int32_t>> send, recv;
};

// First tree cell of every base cell (nbase + 1 entries, the last = cells).
// Returns false if the tree's order does not visit base cells in ascending
// lexicographic order.
bool base_starts(const Tree& t, std::vector<int64_t>* starts);

// nranks contiguous ranges of base cells whose cell counts are as even as the
// base-cell granularity allows (each range holds at least one base cell).
// Returns false if nranks exceeds the number of base cells.
bool balanced_cuts(const std::vector<int64_t>& starts, int nranks, std::vector<int64_t>* base_cut);

// The sub-domain of `rank` under base_cut: owned cells, ghosts (every cell
// sharing a conforming face or a parent face family with an owned cell),
// local face lists, the skeleton (the tree's skeleton cells and the cells
// whose face data a neighbour receives) and the exchange lists.
void build_subdomain(const Tree& t, const std::vector<int64_t>& starts,
                     const std::vector<int64_t>& base_cut, int rank, SubDomain* out);

}  // namespace ader
