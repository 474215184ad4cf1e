// Host-side 3^d spacetree: leaves, face lists, skeleton/enclave split and
// remeshing plans for the ADER-DG step (paper Sec. 2.3 and Sec. 3).
//
// A cell is (level, i_x, i_y, i_z) on the periodic grid of base[d] * 3^level
// cells per axis.  The tree is the set of leaves plus the set of refined
// (inner) nodes.  Cells are numbered in depth-first order of the tree (base
// cells lexicographic with x fastest, children likewise); the skeleton and
// enclave batches are index lists into that numbering.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ader {

struct Key {
  int level;
  int x[3];
};

uint64_t pack(const Key& k);
Key unpack(uint64_t v);

// Open-addressing hash table from packed cell keys to int32 values (linear
// probing, power-of-two capacity, splitmix64 mixing of the key, tombstones on
// erase).  The tree's hot operations are lookups of packed keys; this keeps
// them to one or two cache lines each.  The two all-ones patterns mark empty
// and erased slots (a packed key's top nibble holds a level <= 7).
class KeyMap {
 public:
  explicit KeyMap(size_t expect = 16) { reset(expect); }
  void reset(size_t expect) {
    size_t cap = 16;
    while (cap < 2 * expect) cap <<= 1;
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, 0);
    size_ = used_ = 0;
  }
  size_t size() const { return size_; }
  // returns true when k was not present
  bool insert(uint64_t k, int32_t v = 0) {
    if (2 * (used_ + 1) > keys_.size()) grow();
    size_t i = slot(k), tomb = SIZE_MAX;
    for (;; i = (i + 1) & (keys_.size() - 1)) {
      if (keys_[i] == k) return false;
      if (keys_[i] == kErased && tomb == SIZE_MAX) tomb = i;
      if (keys_[i] == kEmpty) break;
    }
    if (tomb != SIZE_MAX) {
      i = tomb;
    } else {
      ++used_;
    }
    keys_[i] = k;
    vals_[i] = v;
    ++size_;
    return true;
  }
  const int32_t* find(uint64_t k) const {
    for (size_t i = slot(k);; i = (i + 1) & (keys_.size() - 1)) {
      if (keys_[i] == k) return &vals_[i];
      if (keys_[i] == kEmpty) return nullptr;
    }
  }
  int32_t* find_mut(uint64_t k) { return const_cast<int32_t*>(static_cast<const KeyMap*>(this)->find(k)); }
  bool count(uint64_t k) const { return find(k) != nullptr; }
  void erase(uint64_t k) {
    for (size_t i = slot(k);; i = (i + 1) & (keys_.size() - 1)) {
      if (keys_[i] == k) {
        keys_[i] = kErased;
        --size_;
        return;
      }
      if (keys_[i] == kEmpty) return;
    }
  }
  template <class F>
  void for_each(F&& f) const {
    for (size_t i = 0; i < keys_.size(); ++i)
      if (keys_[i] != kEmpty && keys_[i] != kErased) f(keys_[i], vals_[i]);
  }

 private:
  static constexpr uint64_t kEmpty = ~uint64_t(0);
  static constexpr uint64_t kErased = ~uint64_t(0) - 1;
  size_t slot(uint64_t k) const {
    k += 0x9e3779b97f4a7c15ull;  // splitmix64 finaliser
    k = (k ^ (k >> 30)) * 0xbf58476d1ce4e5b9ull;
    k = (k ^ (k >> 27)) * 0x94d049bb133111ebull;
    return size_t(k ^ (k >> 31)) & (keys_.size() - 1);
  }
  void grow() {
    std::vector<uint64_t> ok;
    std::vector<int32_t> ov;
    ok.swap(keys_);
    ov.swap(vals_);
    reset(size_ > 8 ? 2 * size_ : 16);
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty && ok[i] != kErased) insert(ok[i], ov[i]);
  }
  std::vector<uint64_t> keys_;
  std::vector<int32_t> vals_;
  size_t size_ = 0, used_ = 0;
};

// One transition: the coarse cell's face (dir, coarse_side) is split into
// 3^(d-1) child faces; child sigma (lowest tangential direction fastest)
// belongs to fine cell child_fine[parent * 3^(d-1) + sigma].
struct ParentFace {
  int32_t coarse;
  int32_t dir;
  int32_t coarse_side;  // 0: the coarse cell's -dir face, 1: its +dir face
  int32_t pad;
};

struct ConfFace {
  int32_t left;   // cell whose +dir face this is
  int32_t right;  // cell whose -dir face this is
  int32_t dir;
  int32_t pad;
};

// How a cell of the new mesh gets its data during a remesh.
struct TransferItem {
  int32_t kind;   // 0 copy, 1 interpolate from parent, 2 project from children
  int32_t src;    // old cell index (kinds 0, 1) or offset into child list (kind 2)
  int32_t child;  // kind 1: child position s_x + 3 s_y + 9 s_z inside the parent
  int32_t pad;
};

// The lists a device step launches over, in one cell numbering: the whole
// mesh (Tree) or one sub-domain of a partition (SubDomain).  Cells
// [0, nowned) are predicted and corrected; cells [nowned, nlocal) are ghosts
// whose face data arrive by exchange (none outside a partition).
struct MeshLists {
  int64_t nlocal = 0, nowned = 0;
  std::vector<int8_t> levels;             // per local cell

  // Skeleton/enclave split: skel_cells + encl_cells partition [0, nowned).
  // conf: the conforming faces, those whose two cells are both skeleton
  // first (n_conf_skeleton of them).
  std::vector<int32_t> skel_cells, encl_cells;
  std::vector<ConfFace> conf;
  int64_t n_conf_skeleton = 0;
  std::vector<ParentFace> parents;
  std::vector<int32_t> child_fine;

  // Enclave pipeline of a step (Tree::set_chunks(K), recomputed by
  // classify()): the enclave cells split into K contiguous chunks
  // encl_cells[chunk_off[k] .. chunk_off[k+1]); the conforming faces after
  // the skeleton ones ordered by the chunk whose predictor completes their two
  // cells, conf[n_conf_skeleton + face_off[k] .. n_conf_skeleton +
  // face_off[k+1]); and every cell in corr_cells, grouped by the stage after
  // which all its face fluxes exist: group 0 after the skeleton tasks, group
  // k + 1 after chunk k (corr_cells[corr_off[g] .. corr_off[g+1])).
  int chunks = 1;
  std::vector<int64_t> chunk_off, face_off, corr_off;
  std::vector<int32_t> corr_cells;
};

class Tree : public MeshLists {
 public:
  Tree() = default;
  Tree(int dim, const int base[3], int max_level);

  int dim() const { return dim_; }
  int max_level() const { return max_level_; }
  const int* base() const { return base_; }
  int64_t dims(int level, int d) const;

  // The ordered cell list and its derived structures.  Rebuilt by build().
  std::vector<Key> cells;
  std::vector<uint8_t> transition;        // per cell: touches a resolution transition
  std::vector<ConfFace> conf_all;         // conforming faces, build order

  // Skeleton/enclave split (classify()): skeleton = transition cells plus
  // cells flagged for refinement.  conf (MeshLists) is conf_all with the
  // faces whose two cells are both skeleton first.
  std::vector<uint8_t> skeleton;
  void set_chunks(int K);

  // Rebuild order and faces.  Returns false and sets error() if the mesh is
  // not 2:1 balanced.  Leaves the split as transition cells only.
  bool build();
  // Recompute the split; refine_flags (per cell, may be null) adds cells with
  // a positive flag to the skeleton.
  void classify(const int8_t* refine_flags);

  // Apply per-cell flags (+1 refine, -1 coarsen, 0 keep) in the order of
  // `cells`.  Fills the transfer plan for the new order (and the child list
  // for projections).  Calls build() on the new mesh.
  bool remesh(const int8_t* flags, std::vector<TransferItem>* plan,
              std::vector<int32_t>* coarsen_children);

  // Refinement around troubled cells (limiter): +1 for cells with
  // troubled[c] != 0 and their face neighbours (conforming, finer across a
  // parent face, coarser across a child face) below max_level, -1 for every
  // other cell above level 0.
  void refine_around(const uint8_t* troubled, int8_t* flags) const;

  // Geometric criterion around a ball (periodic distance): refine leaves
  // below max_level whose box meets the ball, coarsen leaves above level 0
  // whose parent's box misses it.
  void sphere_flags(const double center[3], double radius, const double lo[3],
                    const double hi[3], int8_t* flags) const;

  const std::string& error() const { return error_; }

  // The adaptive state of the tree: its leaves, the refine flags of its
  // split and the chunk count.  The refined set (the leaves' ancestors) and
  // every list follow from it, so it is a much cheaper undo point than a copy
  // of the whole tree.
  struct State {
    std::vector<Key> leaves;
    std::vector<int8_t> refine_flags;
    int chunks = 1;
  };
  State save() const;
  // Back to a saved state of a balanced mesh: the leaf and refined sets, then
  // build() and the split.
  void restore(State&& s);

 private:
  bool is_leaf(const Key& k) const { return leaves_.count(pack(k)) != 0; }
  bool is_refined(const Key& k) const { return refined_.count(pack(k)) != 0; }
  Key neighbor(const Key& k, int dir, int side) const;
  Key parent(const Key& k) const;
  Key child(const Key& k, const int s[3]) const;
  void touching_children(const Key& k, int dir, int side, std::vector<Key>* out) const;
  int max_level_across(const Key& k, int dir, int side) const;
  int max_level_below_face(const Key& k, int dir, int side) const;
  void split(const Key& k);
  // Depth-first leaf order from the base cells; stores each leaf's position
  // as its value in leaves_ (the index lookups of build() and remesh()).
  void order_cells(std::vector<Key>* out);
  void dfs(const Key& k, std::vector<Key>* out, std::vector<int32_t*>* slots);
  bool plan_by_walk(const std::vector<Key>& old_cells, std::vector<TransferItem>* plan,
                    std::vector<int32_t>* coarsen_children) const;

  int dim_ = 0;
  int base_[3] = {1, 1, 1};
  int max_level_ = 0;
  KeyMap leaves_;   // leaf keys -> position in `cells` (set by build())
  KeyMap refined_;  // keys of refined (non-leaf) nodes, kept in step with leaves_
  std::string error_;
};

}  // namespace ader
