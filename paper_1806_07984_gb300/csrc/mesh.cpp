// Host-side 3^d spacetree (paper Sec. 2.3: three-partitioning on a conformal
// base grid; virtual cells and parent/child faces at resolution transitions;
// Sec. 3 and 3.1: skeleton cells adjacent to a resolution transition).
#include "mesh.h"

#include <algorithm>
#include <cmath>
#include <thread>

namespace ader {

uint64_t pack(const Key& k) {
  return (uint64_t(k.level) << 60) | (uint64_t(k.x[0] & 0xFFFFF) << 40) |
         (uint64_t(k.x[1] & 0xFFFFF) << 20) | uint64_t(k.x[2] & 0xFFFFF);
}

Key unpack(uint64_t v) {
  Key k;
  k.level = int(v >> 60);
  k.x[0] = int((v >> 40) & 0xFFFFF);
  k.x[1] = int((v >> 20) & 0xFFFFF);
  k.x[2] = int(v & 0xFFFFF);
  return k;
}

Tree::Tree(int dim, const int base[3], int max_level) : dim_(dim), max_level_(max_level) {
  for (int d = 0; d < 3; ++d) base_[d] = d < dim ? base[d] : 1;
  for (int z = 0; z < base_[2]; ++z)
    for (int y = 0; y < base_[1]; ++y)
      for (int x = 0; x < base_[0]; ++x) {
        Key k{0, {x, y, z}};
        leaves_.insert(pack(k));
      }
}

int64_t Tree::dims(int level, int d) const {
  int64_t n = base_[d];
  if (d >= dim_) return 1;
  for (int l = 0; l < level; ++l) n *= 3;
  return n;
}

Key Tree::neighbor(const Key& k, int dir, int side) const {
  Key n = k;
  const int64_t m = dims(k.level, dir);
  int64_t c = k.x[dir] + (side == 1 ? 1 : -1);
  c = ((c % m) + m) % m;
  n.x[dir] = int(c);
  return n;
}

Key Tree::parent(const Key& k) const {
  Key p = k;
  p.level = k.level - 1;
  for (int d = 0; d < dim_; ++d) p.x[d] = k.x[d] / 3;
  return p;
}

Key Tree::child(const Key& k, const int s[3]) const {
  Key c = k;
  c.level = k.level + 1;
  for (int d = 0; d < dim_; ++d) c.x[d] = 3 * k.x[d] + s[d];
  return c;
}

// Children of node k touching its face (dir, side), in sub-face order sigma
// (tangential directions ascending, lowest fastest).
void Tree::touching_children(const Key& k, int dir, int side, std::vector<Key>* out) const {
  out->clear();
  int tang[2] = {0, 0}, nt = 0;
  for (int d = 0; d < dim_; ++d)
    if (d != dir) tang[nt++] = d;
  const int count = dim_ == 3 ? 9 : 3;
  for (int sigma = 0; sigma < count; ++sigma) {
    int s[3] = {0, 0, 0};
    s[dir] = side == 0 ? 0 : 2;
    s[tang[0]] = sigma % 3;
    if (nt > 1) s[tang[1]] = sigma / 3;
    out->push_back(child(k, s));
  }
}

int Tree::max_level_below_face(const Key& k, int dir, int side) const {
  if (is_leaf(k)) return k.level;
  int best = k.level;
  std::vector<Key> kids;
  touching_children(k, dir, side, &kids);
  for (const Key& c : kids) best = std::max(best, max_level_below_face(c, dir, side));
  return best;
}

int Tree::max_level_across(const Key& k, int dir, int side) const {
  Key nb = neighbor(k, dir, side);
  if (is_leaf(nb)) return nb.level;
  if (is_refined(nb)) return max_level_below_face(nb, dir, 1 - side);
  return k.level - 1;
}

void Tree::split(const Key& k) {
  leaves_.erase(pack(k));
  refined_.insert(pack(k));
  const int nz = dim_ == 3 ? 3 : 1;
  for (int sz = 0; sz < nz; ++sz)
    for (int sy = 0; sy < 3; ++sy)
      for (int sx = 0; sx < 3; ++sx) {
        int s[3] = {sx, sy, sz};
        leaves_.insert(pack(child(k, s)));
      }
}

void Tree::rebuild_refined() {
  refined_.reset(leaves_.size() / 2 + 16);
  leaves_.for_each([&](uint64_t v, int32_t) {
    Key k = unpack(v);
    while (k.level > 0) {
      k = parent(k);
      if (!refined_.insert(pack(k))) break;
    }
  });
}

void Tree::dfs(const Key& k, std::vector<Key>* out) const {
  if (is_leaf(k)) {
    out->push_back(k);
    return;
  }
  if (!is_refined(k)) return;
  const int nz = dim_ == 3 ? 3 : 1;
  for (int sz = 0; sz < nz; ++sz)
    for (int sy = 0; sy < 3; ++sy)
      for (int sx = 0; sx < 3; ++sx) {
        int s[3] = {sx, sy, sz};
        dfs(child(k, s), out);
      }
}

void Tree::order_cells(std::vector<Key>* out) const {
  out->clear();
  out->reserve(leaves_.size());
  for (int z = 0; z < base_[2]; ++z)
    for (int y = 0; y < base_[1]; ++y)
      for (int x = 0; x < base_[0]; ++x) dfs(Key{0, {x, y, z}}, out);
}

bool Tree::build() {
  order_cells(&cells);
  const int64_t n = int64_t(cells.size());
  KeyMap pos(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) pos.insert(pack(cells[size_t(i)]), int32_t(i));
  conf_all.clear();
  parents.clear();
  child_fine.clear();
  transition.assign(size_t(n), 0);
  // Faces of contiguous cell ranges in parallel (read-only lookups); the
  // per-range lists are concatenated in range order, so the result equals
  // the sequential sweep.
  struct Part {
    std::vector<ConfFace> conf;
    std::vector<ParentFace> parents;
    std::vector<int32_t> child_fine, marked;
    bool ok = true;
  };
  const int nt = int(std::max<int64_t>(1, std::min<int64_t>(
      int64_t(std::max(1u, std::thread::hardware_concurrency())), std::min<int64_t>(16, n / 4096))));
  std::vector<Part> parts(static_cast<size_t>(nt));
  auto sweep = [&](int t) {
    Part& P = parts[size_t(t)];
    std::vector<Key> kids;
    const int64_t b = n * t / nt, e = n * (t + 1) / nt;
    for (int64_t i = b; i < e && P.ok; ++i) {
      const Key k = cells[size_t(i)];
      for (int dir = 0; dir < dim_; ++dir) {
        for (int side = 1; side >= 0; --side) {
          Key nb = neighbor(k, dir, side);
          if (side == 1 && is_leaf(nb)) {
            P.conf.push_back({int32_t(i), *pos.find(pack(nb)), dir, 0});
          } else if (is_refined(nb)) {
            touching_children(nb, dir, 1 - side, &kids);
            P.parents.push_back({int32_t(i), dir, side, 0});
            for (const Key& c : kids) {
              const int32_t* it = pos.find(pack(c));
              if (!it) {
                P.ok = false;
                break;
              }
              P.child_fine.push_back(*it);
              P.marked.push_back(*it);
            }
            P.marked.push_back(int32_t(i));
          }
        }
      }
    }
  };
  std::vector<std::thread> workers;
  for (int t = 1; t < nt; ++t) workers.emplace_back(sweep, t);
  sweep(0);
  for (std::thread& w : workers) w.join();
  for (const Part& P : parts) {
    if (!P.ok) {
      error_ = "mesh is not 2:1 balanced";
      return false;
    }
    conf_all.insert(conf_all.end(), P.conf.begin(), P.conf.end());
    parents.insert(parents.end(), P.parents.begin(), P.parents.end());
    child_fine.insert(child_fine.end(), P.child_fine.begin(), P.child_fine.end());
    for (int32_t c : P.marked) transition[size_t(c)] = 1;
  }
  classify(nullptr);
  error_.clear();
  return true;
}

void Tree::classify(const int8_t* refine_flags) {
  const size_t n = cells.size();
  skeleton.assign(n, 0);
  skel_cells.clear();
  encl_cells.clear();
  for (size_t i = 0; i < n; ++i) {
    skeleton[i] = transition[i] || (refine_flags && refine_flags[i] > 0);
    (skeleton[i] ? skel_cells : encl_cells).push_back(int32_t(i));
  }
  conf.clear();
  conf.reserve(conf_all.size());
  for (int pass = 0; pass < 2; ++pass)
    for (const ConfFace& f : conf_all) {
      const bool both = skeleton[size_t(f.left)] && skeleton[size_t(f.right)];
      if (both == (pass == 0)) conf.push_back(f);
    }
  n_conf_skeleton = 0;
  for (const ConfFace& f : conf_all)
    n_conf_skeleton += (skeleton[size_t(f.left)] && skeleton[size_t(f.right)]) ? 1 : 0;
  // enclave pipeline: chunk of every cell (-1 = skeleton), faces by the later
  // chunk of their two cells, cells by the latest chunk among their faces
  const int K = std::max(1, chunks);
  const int64_t ne = int64_t(encl_cells.size());
  std::vector<int> chunk_of(n, -1);
  chunk_off.assign(size_t(K) + 1, 0);
  for (int k = 0; k <= K; ++k) chunk_off[size_t(k)] = ne * k / K;
  for (int k = 0; k < K; ++k)
    for (int64_t p = chunk_off[size_t(k)]; p < chunk_off[size_t(k) + 1]; ++p)
      chunk_of[size_t(encl_cells[size_t(p)])] = k;
  std::vector<int> ready(n);
  for (size_t i = 0; i < n; ++i) ready[i] = chunk_of[i];
  std::vector<std::vector<ConfFace>> by_chunk(static_cast<size_t>(K));
  for (size_t i = size_t(n_conf_skeleton); i < conf.size(); ++i) {
    const ConfFace& f = conf[i];
    const int r = std::max(chunk_of[size_t(f.left)], chunk_of[size_t(f.right)]);
    by_chunk[size_t(r)].push_back(f);
    ready[size_t(f.left)] = std::max(ready[size_t(f.left)], r);
    ready[size_t(f.right)] = std::max(ready[size_t(f.right)], r);
  }
  face_off.assign(size_t(K) + 1, 0);
  size_t pos = size_t(n_conf_skeleton);
  for (int k = 0; k < K; ++k) {
    for (const ConfFace& f : by_chunk[size_t(k)]) conf[pos++] = f;
    face_off[size_t(k) + 1] = int64_t(pos) - n_conf_skeleton;
  }
  corr_off.assign(size_t(K) + 2, 0);
  for (size_t i = 0; i < n; ++i) ++corr_off[size_t(ready[i] + 1) + 1];
  for (int g = 0; g <= K; ++g) corr_off[size_t(g) + 1] += corr_off[size_t(g)];
  corr_cells.assign(n, 0);
  std::vector<int64_t> fill(corr_off.begin(), corr_off.end() - 1);
  for (size_t i = 0; i < n; ++i) corr_cells[size_t(fill[size_t(ready[i] + 1)]++)] = int32_t(i);
}

void Tree::refine_around(const uint8_t* troubled, int8_t* flags) const {
  const size_t n = cells.size();
  std::vector<uint8_t> mark(troubled, troubled + n);
  for (const ConfFace& f : conf_all) {
    if (troubled[size_t(f.left)]) mark[size_t(f.right)] = 1;
    if (troubled[size_t(f.right)]) mark[size_t(f.left)] = 1;
  }
  const size_t S = dim_ == 3 ? 9 : 3;
  for (size_t p = 0; p < parents.size(); ++p) {
    const size_t coarse = size_t(parents[p].coarse);
    for (size_t s = 0; s < S; ++s) {
      const size_t fine = size_t(child_fine[p * S + s]);
      if (troubled[coarse]) mark[fine] = 1;
      if (troubled[fine]) mark[coarse] = 1;
    }
  }
  for (size_t i = 0; i < n; ++i) {
    const int lv = cells[i].level;
    flags[i] = mark[i] ? (lv < max_level_ ? 1 : 0) : (lv > 0 ? -1 : 0);
  }
}

void Tree::set_chunks(int K) {
  chunks = std::max(1, K);
  std::vector<int8_t> flags(cells.size(), 0);
  for (size_t i = 0; i < cells.size(); ++i) flags[i] = (skeleton[i] && !transition[i]) ? 1 : 0;
  classify(flags.data());
}

bool Tree::remesh(const int8_t* flags, std::vector<TransferItem>* plan,
                  std::vector<int32_t>* coarsen_children) {
  const std::vector<Key> old_cells = cells;
  KeyMap old_index(old_cells.size());
  for (size_t i = 0; i < old_cells.size(); ++i) old_index.insert(pack(old_cells[i]), int32_t(i));
  KeyMap coarsen;
  // 1. refine flagged leaves below max_level
  std::vector<Key> split_queue;
  for (size_t i = 0; i < old_cells.size(); ++i) {
    const Key& k = old_cells[i];
    if (flags[i] < 0 && k.level > 0) coarsen.insert(pack(k));
    if (flags[i] > 0 && k.level < max_level_) {
      split(k);
      split_queue.push_back(k);
    }
  }
  // 2. 2:1 face balance to a fixpoint.  Splitting a cell of level L puts
  // leaves of level L+1 on its faces, which violates the rule only for a
  // leaf of level <= L-1 across one of them: the leaf covering the
  // neighbour position.  A worklist over the splits reaches the same (unique,
  // smallest) balanced refinement as sweeping all leaves until nothing changes.
  while (!split_queue.empty()) {
    const Key c = split_queue.back();
    split_queue.pop_back();
    for (int dir = 0; dir < dim_; ++dir)
      for (int side = 0; side < 2; ++side)
        for (;;) {  // a split cover may leave a child that is still too coarse
          Key cover = neighbor(c, dir, side);
          while (cover.level > 0 && !is_leaf(cover)) cover = parent(cover);
          if (!is_leaf(cover) || cover.level + 2 > c.level + 1) break;
          split(cover);
          split_queue.push_back(cover);
        }
  }
  rebuild_refined();
  // 3. coarsen complete families of flagged leaves whose parent stays balanced
  std::vector<uint64_t> fams;
  coarsen.for_each([&](uint64_t v, int32_t) {
    Key k = unpack(v);
    if (is_leaf(k)) fams.push_back(pack(parent(k)));
  });
  std::sort(fams.begin(), fams.end());
  fams.erase(std::unique(fams.begin(), fams.end()), fams.end());
  std::vector<Key> approved;
  const int nz = dim_ == 3 ? 3 : 1;
  for (uint64_t v : fams) {
    Key P = unpack(v);
    bool ok = true;
    for (int sz = 0; sz < nz && ok; ++sz)
      for (int sy = 0; sy < 3 && ok; ++sy)
        for (int sx = 0; sx < 3 && ok; ++sx) {
          int s[3] = {sx, sy, sz};
          const uint64_t c = pack(child(P, s));
          if (!leaves_.count(c) || !coarsen.count(c)) ok = false;
        }
    for (int dir = 0; dir < dim_ && ok; ++dir)
      for (int side = 0; side < 2 && ok; ++side)
        if (max_level_across(P, dir, side) >= P.level + 2) ok = false;
    if (ok) approved.push_back(P);
  }
  for (const Key& P : approved) {
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 3; ++sy)
        for (int sx = 0; sx < 3; ++sx) {
          int s[3] = {sx, sy, sz};
          leaves_.erase(pack(child(P, s)));
        }
    leaves_.insert(pack(P));
  }
  rebuild_refined();
  if (!build()) return false;
  // 4. transfer plan for the new order
  plan->clear();
  coarsen_children->clear();
  for (const Key& k : cells) {
    TransferItem t{0, 0, 0, 0};
    const int32_t* it = old_index.find(pack(k));
    if (it) {
      t.kind = 0;
      t.src = *it;
    } else if (k.level > 0 && old_index.count(pack(parent(k)))) {
      Key p = parent(k);
      t.kind = 1;
      t.src = *old_index.find(pack(p));
      int s[3] = {0, 0, 0};
      for (int d = 0; d < dim_; ++d) s[d] = k.x[d] - 3 * p.x[d];
      t.child = s[0] + 3 * s[1] + 9 * s[2];
    } else {
      t.kind = 2;
      t.src = int32_t(coarsen_children->size());
      for (int sz = 0; sz < nz; ++sz)
        for (int sy = 0; sy < 3; ++sy)
          for (int sx = 0; sx < 3; ++sx) {
            int s[3] = {sx, sy, sz};
            const int32_t* c = old_index.find(pack(child(k, s)));
            if (!c) {
              error_ = "remesh changed a cell by more than one level";
              return false;
            }
            coarsen_children->push_back(*c);
          }
    }
    plan->push_back(t);
  }
  return true;
}

void Tree::sphere_flags(const double center[3], double radius, const double lo[3],
                        const double hi[3], int8_t* flags) const {
  auto meets = [&](const Key& k) {
    double dist2 = 0.0;
    for (int d = 0; d < dim_; ++d) {
      const double L = hi[d] - lo[d];
      const double h = L / double(dims(k.level, d));
      const double a = lo[d] + double(k.x[d]) * h;
      const double b = a + h;
      double best = -1.0;
      const double shifts[3] = {-L, 0.0, L};
      for (double sh : shifts) {
        const double c = center[d] + sh;
        const double g = std::max(std::max(a - c, 0.0), c - b);
        best = best < 0.0 ? g : std::min(best, g);
      }
      dist2 += best * best;
    }
    return dist2 <= radius * radius;
  };
  for (size_t i = 0; i < cells.size(); ++i) {
    const Key& k = cells[i];
    int8_t f = 0;
    if (k.level < max_level_ && meets(k))
      f = 1;
    else if (k.level > 0 && !meets(parent(k)))
      f = -1;
    flags[i] = f;
  }
}

}  // namespace ader
