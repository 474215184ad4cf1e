// Host-side 3^d spacetree (paper Sec. 2.3: three-partitioning on a conformal
// base grid; virtual cells and parent/child faces at resolution transitions;
// Sec. 3 and 3.1: skeleton cells adjacent to a resolution transition).
#include "mesh.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace ader {

namespace {

// Threads for a host pass over n items: one per 4096 items, at most 16 and
// the hardware's count.
int pass_threads(int64_t n) {
  const int64_t hw = int64_t(std::max(1u, std::thread::hardware_concurrency()));
  return int(std::max<int64_t>(1, std::min<int64_t>(hw, std::min<int64_t>(16, n / 4096))));
}

// f(t, begin, end) on the T contiguous ranges [n t / T, n (t + 1) / T) of
// [0, n), range 0 on the calling thread.
template <class F>
void parallel_ranges(int64_t n, int T, F&& f) {
  std::vector<std::thread> workers;
  for (int t = 1; t < T; ++t) workers.emplace_back([&, t] { f(t, n * t / T, n * (t + 1) / T); });
  f(0, int64_t(0), n / T);
  for (std::thread& w : workers) w.join();
}

}  // namespace

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

void Tree::dfs(const Key& k, std::vector<Key>* out, std::vector<int32_t*>* slots) {
  if (int32_t* pos = leaves_.find_mut(pack(k))) {
    out->push_back(k);
    slots->push_back(pos);
    return;
  }
  if (!is_refined(k)) return;
  const int nz = dim_ == 3 ? 3 : 1;
  for (int sz = 0; sz < nz; ++sz)
    for (int sy = 0; sy < 3; ++sy)
      for (int sx = 0; sx < 3; ++sx) {
        int s[3] = {sx, sy, sz};
        dfs(child(k, s), out, slots);
      }
}

void Tree::order_cells(std::vector<Key>* out) {
  // base cells x fastest, each followed by its subtree.  The refined region
  // is local, so the base cells go in many small contiguous groups, taken by
  // the threads in turn and concatenated in group order.
  const int64_t nb = int64_t(base_[0]) * base_[1] * base_[2];
  const int T = pass_threads(int64_t(leaves_.size()));
  const int64_t G = std::min<int64_t>(nb, int64_t(T) * 64);
  std::vector<std::vector<Key>> part(static_cast<size_t>(G));
  std::vector<std::vector<int32_t*>> slot(static_cast<size_t>(G));
  std::atomic<int64_t> next{0};
  auto work = [&]() {
    for (int64_t g = next++; g < G; g = next++)
      for (int64_t i = nb * g / G; i < nb * (g + 1) / G; ++i) {
        const Key k{0, {int(i % base_[0]), int((i / base_[0]) % base_[1]),
                        int(i / (int64_t(base_[0]) * base_[1]))}};
        dfs(k, &part[size_t(g)], &slot[size_t(g)]);
      }
  };
  parallel_ranges(T, T, [&](int, int64_t, int64_t) { work(); });
  std::vector<size_t> off(static_cast<size_t>(G) + 1, 0);
  for (int64_t g = 0; g < G; ++g) off[size_t(g) + 1] = off[size_t(g)] + part[size_t(g)].size();
  out->resize(off[size_t(G)]);
  parallel_ranges(G, T, [&](int, int64_t b, int64_t e) {
    for (int64_t g = b; g < e; ++g)
      for (size_t i = 0; i < part[size_t(g)].size(); ++i) {
        (*out)[off[size_t(g)] + i] = part[size_t(g)][i];
        *slot[size_t(g)][i] = int32_t(off[size_t(g)] + i);
      }
  });
}

bool Tree::build() {
  order_cells(&cells);  // also sets every leaf's position in leaves_
  const int64_t n = int64_t(cells.size());
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
  const int nt = pass_threads(n);
  std::vector<Part> parts(static_cast<size_t>(nt));
  parallel_ranges(n, nt, [&](int t, int64_t b, int64_t e) {
    Part& P = parts[size_t(t)];
    P.conf.reserve(size_t(e - b) * size_t(dim_));
    std::vector<Key> kids;
    for (int64_t i = b; i < e && P.ok; ++i) {
      const Key k = cells[size_t(i)];
      for (int dir = 0; dir < dim_; ++dir) {
        for (int side = 1; side >= 0; --side) {
          Key nb = neighbor(k, dir, side);
          const uint64_t key = pack(nb);
          // A leaf neighbour of the same level is usually a fixed distance
          // away in the depth-first order (a sibling, or the next base cell):
          // a key compare there saves the hash lookup.
          const int64_t st = k.level > 0 ? (dir == 0 ? 1 : (dir == 1 ? 3 : 9))
                                         : (dir == 0 ? 1 : (dir == 1 ? base_[0] : int64_t(base_[0]) * base_[1]));
          const int64_t cand = side == 1 ? i + st : i - st;
          int32_t at = -1;
          if (cand >= 0 && cand < n && pack(cells[size_t(cand)]) == key) {
            at = int32_t(cand);
          } else if (const int32_t* leaf = leaves_.find(key)) {
            at = *leaf;
          }
          if (at >= 0) {  // a leaf is never refined
            if (side == 1) P.conf.push_back({int32_t(i), at, dir, 0});
          } else if (is_refined(nb)) {
            touching_children(nb, dir, 1 - side, &kids);
            P.parents.push_back({int32_t(i), dir, side, 0});
            for (const Key& c : kids) {
              const int32_t* it = leaves_.find(pack(c));
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
  });
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
  nlocal = nowned = n;
  levels.resize(size_t(n));
  for (int64_t i = 0; i < n; ++i) levels[size_t(i)] = int8_t(cells[size_t(i)].level);
  classify(nullptr);
  error_.clear();
  return true;
}

void Tree::classify(const int8_t* refine_flags) {
  const size_t n = cells.size();
  // The split in contiguous cell ranges: per-range skeleton counts, then each
  // range fills both lists from its own offsets (the lists stay ascending).
  skeleton.assign(n, 0);
  const int Tc = pass_threads(int64_t(n));
  std::vector<int64_t> nsk(size_t(Tc) + 1, 0);
  parallel_ranges(int64_t(n), Tc, [&](int t, int64_t b, int64_t e) {
    int64_t c = 0;
    for (int64_t i = b; i < e; ++i) {
      skeleton[size_t(i)] = transition[size_t(i)] || (refine_flags && refine_flags[i] > 0);
      c += skeleton[size_t(i)];
    }
    nsk[size_t(t) + 1] = c;
  });
  for (int t = 0; t < Tc; ++t) nsk[size_t(t) + 1] += nsk[size_t(t)];
  skel_cells.resize(size_t(nsk[size_t(Tc)]));
  encl_cells.resize(n - size_t(nsk[size_t(Tc)]));
  parallel_ranges(int64_t(n), Tc, [&](int t, int64_t b, int64_t e) {
    int64_t ps = nsk[size_t(t)], pe = b - nsk[size_t(t)];
    for (int64_t i = b; i < e; ++i) {
      if (skeleton[size_t(i)])
        skel_cells[size_t(ps++)] = int32_t(i);
      else
        encl_cells[size_t(pe++)] = int32_t(i);
    }
  });
  // enclave pipeline: chunk of every cell (-1 = skeleton), faces by the later
  // chunk of their two cells, cells by the latest chunk among their faces.
  // conf = the faces with two skeleton cells (conf_all order), then the
  // others grouped by that chunk (conf_all order within a group).
  const int K = std::max(1, chunks);
  const int64_t ne = int64_t(encl_cells.size());
  std::vector<int> chunk_of(n, -1);
  chunk_off.assign(size_t(K) + 1, 0);
  for (int k = 0; k <= K; ++k) chunk_off[size_t(k)] = ne * k / K;
  for (int k = 0; k < K; ++k)
    for (int64_t p = chunk_off[size_t(k)]; p < chunk_off[size_t(k) + 1]; ++p)
      chunk_of[size_t(encl_cells[size_t(p)])] = k;
  std::vector<int> ready(chunk_of);
  const size_t nf = conf_all.size();
  std::vector<int> group(nf);  // -1: both cells skeleton, else the face's chunk
  // Faces in T contiguous ranges: groups, per-range counts, and each cell's
  // latest face chunk (a maximum, so the order of the updates does not
  // matter); then every range scatters its faces from its own offset in each
  // group, which keeps conf_all order within a group as a sequential pass.
  const int T = pass_threads(int64_t(nf));
  std::vector<std::vector<int64_t>> cnt(size_t(T), std::vector<int64_t>(size_t(K) + 1, 0));
  auto raise = [](int* p, int r) {
    int cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (cur < r && !__atomic_compare_exchange_n(p, &cur, r, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
  };
  parallel_ranges(int64_t(nf), T, [&](int t, int64_t b, int64_t e) {
    std::vector<int64_t>& C = cnt[size_t(t)];
    for (int64_t f = b; f < e; ++f) {
      const ConfFace& F = conf_all[size_t(f)];
      const int r = std::max(chunk_of[size_t(F.left)], chunk_of[size_t(F.right)]);
      group[size_t(f)] = r;
      ++C[size_t(r + 1)];
      if (r >= 0) {
        raise(&ready[size_t(F.left)], r);
        raise(&ready[size_t(F.right)], r);
      }
    }
  });
  std::vector<int64_t> count(size_t(K) + 1, 0);
  for (int t = 0; t < T; ++t)
    for (int g = 0; g <= K; ++g) count[size_t(g)] += cnt[size_t(t)][size_t(g)];
  n_conf_skeleton = count[0];
  face_off.assign(size_t(K) + 1, 0);
  for (int k = 0; k < K; ++k) face_off[size_t(k) + 1] = face_off[size_t(k)] + count[size_t(k) + 1];
  std::vector<int64_t> put(size_t(K) + 1);
  put[0] = 0;
  for (int k = 0; k < K; ++k) put[size_t(k) + 1] = n_conf_skeleton + face_off[size_t(k)];
  for (int t = 0; t < T; ++t)  // cnt[t] becomes range t's first slot in each group
    for (int g = 0; g <= K; ++g) {
      const int64_t c = cnt[size_t(t)][size_t(g)];
      cnt[size_t(t)][size_t(g)] = put[size_t(g)];
      put[size_t(g)] += c;
    }
  conf.resize(nf);
  parallel_ranges(int64_t(nf), T, [&](int t, int64_t b, int64_t e) {
    std::vector<int64_t>& at = cnt[size_t(t)];
    for (int64_t f = b; f < e; ++f) conf[size_t(at[size_t(group[size_t(f)] + 1)]++)] = conf_all[size_t(f)];
  });
  // corrector groups: the same two-pass scheme over cell ranges
  std::vector<std::vector<int64_t>> gc(size_t(Tc), std::vector<int64_t>(size_t(K) + 1, 0));
  parallel_ranges(int64_t(n), Tc, [&](int t, int64_t b, int64_t e) {
    std::vector<int64_t>& C = gc[size_t(t)];
    for (int64_t i = b; i < e; ++i) ++C[size_t(ready[size_t(i)] + 1)];
  });
  corr_off.assign(size_t(K) + 2, 0);
  for (int t = 0; t < Tc; ++t)
    for (int g = 0; g <= K; ++g) corr_off[size_t(g) + 1] += gc[size_t(t)][size_t(g)];
  for (int g = 0; g <= K; ++g) corr_off[size_t(g) + 1] += corr_off[size_t(g)];
  std::vector<int64_t> at(corr_off.begin(), corr_off.end() - 1);
  for (int t = 0; t < Tc; ++t)  // gc[t] becomes range t's first slot in each group
    for (int g = 0; g <= K; ++g) {
      const int64_t c = gc[size_t(t)][size_t(g)];
      gc[size_t(t)][size_t(g)] = at[size_t(g)];
      at[size_t(g)] += c;
    }
  corr_cells.assign(n, 0);
  parallel_ranges(int64_t(n), Tc, [&](int t, int64_t b, int64_t e) {
    std::vector<int64_t>& A = gc[size_t(t)];
    for (int64_t i = b; i < e; ++i) corr_cells[size_t(A[size_t(ready[size_t(i)] + 1)]++)] = int32_t(i);
  });
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

Tree::State Tree::save() const {
  State s{cells, std::vector<int8_t>(cells.size(), 0), chunks};
  for (size_t i = 0; i < cells.size(); ++i) s.refine_flags[i] = (skeleton[i] && !transition[i]) ? 1 : 0;
  return s;
}

void Tree::restore(State&& s) {
  leaves_.reset(s.leaves.size());
  refined_.reset(s.leaves.size() / 8 + 16);
  for (const Key& k : s.leaves) {
    leaves_.insert(pack(k));
    for (Key p = k; p.level > 0;) {  // ancestors up to the first one already known
      p = parent(p);
      if (!refined_.insert(pack(p))) break;
    }
  }
  chunks = s.chunks;
  build();
  classify(s.refine_flags.data());
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
  // 3. coarsen complete families of flagged leaves whose parent stays balanced
  std::vector<uint64_t> fams;
  coarsen.for_each([&](uint64_t v, int32_t) {
    Key k = unpack(v);
    if (is_leaf(k)) fams.push_back(pack(parent(k)));
  });
  std::sort(fams.begin(), fams.end());
  fams.erase(std::unique(fams.begin(), fams.end()), fams.end());
  // the checks only read the sets: families in parallel ranges, applied in order
  std::vector<uint8_t> ok_fam(fams.size(), 0);
  const int nz = dim_ == 3 ? 3 : 1;
  parallel_ranges(int64_t(fams.size()), pass_threads(int64_t(fams.size()) * 32), [&](int, int64_t b, int64_t e) {
    for (int64_t f = b; f < e; ++f) {
      const Key P = unpack(fams[size_t(f)]);
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
      ok_fam[size_t(f)] = ok ? 1 : 0;
    }
  });
  std::vector<Key> approved;
  for (size_t f = 0; f < fams.size(); ++f)
    if (ok_fam[f]) approved.push_back(unpack(fams[f]));
  for (const Key& P : approved) {
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 3; ++sy)
        for (int sx = 0; sx < 3; ++sx) {
          int s[3] = {sx, sy, sz};
          leaves_.erase(pack(child(P, s)));
        }
    leaves_.insert(pack(P));
    refined_.erase(pack(P));
  }
  if (!build()) return false;
  // 4. transfer plan for the new order
  if (plan_by_walk(old_cells, plan, coarsen_children)) return true;
  KeyMap old_index(old_cells.size());
  for (size_t i = 0; i < old_cells.size(); ++i) old_index.insert(pack(old_cells[i]), int32_t(i));
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

// Both cell lists are depth-first orders of the same base grid, and a remesh
// changes cells by one level at most: the new list is the old one with every
// refined leaf replaced in place by its 3^d children (lexicographic, x
// fastest) and every coarsened family by its parent.  One merge walk over the
// two lists therefore finds the source of every new cell; each entry is
// checked against the keys, and the walk reports failure (the caller then
// uses key lookups) on anything else.
bool Tree::plan_by_walk(const std::vector<Key>& old_cells, std::vector<TransferItem>* plan,
                        std::vector<int32_t>* coarsen_children) const {
  plan->clear();
  coarsen_children->clear();
  plan->reserve(cells.size());
  const int nz = dim_ == 3 ? 3 : 1;
  const int fam = 9 * nz;
  const size_t no = old_cells.size();
  size_t j = 0;
  for (const Key& k : cells) {
    if (j >= no) return false;
    const Key& o = old_cells[j];
    TransferItem t{0, 0, 0, 0};
    if (pack(k) == pack(o)) {
      t.src = int32_t(j++);
    } else if (k.level == o.level + 1 && pack(parent(k)) == pack(o)) {
      t.kind = 1;
      t.src = int32_t(j);
      int s[3] = {0, 0, 0};
      for (int d = 0; d < dim_; ++d) s[d] = k.x[d] - 3 * o.x[d];
      t.child = s[0] + 3 * s[1] + 9 * s[2];
      if (t.child == fam - 1) ++j;  // the parent's last child in the order
    } else if (o.level == k.level + 1 && j + size_t(fam) <= no) {
      t.kind = 2;
      t.src = int32_t(coarsen_children->size());
      for (int sz = 0; sz < nz; ++sz)
        for (int sy = 0; sy < 3; ++sy)
          for (int sx = 0; sx < 3; ++sx) {
            int s[3] = {sx, sy, sz};
            if (pack(old_cells[j]) != pack(child(k, s))) return false;
            coarsen_children->push_back(int32_t(j++));
          }
    } else {
      return false;
    }
    plan->push_back(t);
  }
  return j == no;
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
  const int64_t n = int64_t(cells.size());
  parallel_ranges(n, pass_threads(n), [&](int, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const Key& k = cells[size_t(i)];
      int8_t f = 0;
      if (k.level < max_level_ && meets(k))
        f = 1;
      else if (k.level > 0 && !meets(parent(k)))
        f = -1;
      flags[i] = f;
    }
  });
}

}  // namespace ader
