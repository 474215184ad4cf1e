// Sub-domains of the depth-first cell order (see partition.h).
#include "partition.h"

#include <algorithm>
#include <cmath>

namespace ader {

bool base_starts(const Tree& t, std::vector<int64_t>* starts) {
  const int D = t.dim();
  const int* b = t.base();
  const int64_t nbase = int64_t(b[0]) * b[1] * b[2];
  std::vector<int64_t> count(size_t(nbase) + 1, 0);
  int64_t prev = -1;
  for (const Key& k : t.cells) {
    int64_t scale = 1;
    for (int l = 0; l < k.level; ++l) scale *= 3;
    int64_t idx = 0, stride = 1;
    for (int d = 0; d < D; ++d) {
      idx += (k.x[d] / scale) * stride;
      stride *= b[d];
    }
    if (idx < prev || idx >= nbase) return false;
    prev = idx;
    ++count[size_t(idx) + 1];
  }
  for (int64_t i = 0; i < nbase; ++i) count[size_t(i) + 1] += count[size_t(i)];
  starts->swap(count);
  return true;
}

bool balanced_cuts(const std::vector<int64_t>& starts, int nranks, std::vector<int64_t>* base_cut) {
  const int64_t nbase = int64_t(starts.size()) - 1;
  if (nranks < 1 || nranks > nbase) return false;
  const int64_t C = starts.back();
  base_cut->assign(size_t(nranks) + 1, 0);
  (*base_cut)[size_t(nranks)] = nbase;
  for (int k = 1; k < nranks; ++k) {
    const double target = double(C) * k / nranks;
    const int64_t lo = (*base_cut)[size_t(k) - 1] + 1;  // at least one base cell per range
    const int64_t hi = nbase - (nranks - k);
    int64_t b = int64_t(std::lower_bound(starts.begin(), starts.end(), int64_t(target + 0.5)) -
                        starts.begin());
    if (b > lo && std::abs(double(starts[size_t(b) - 1]) - target) <= std::abs(double(starts[size_t(b)]) - target))
      --b;
    (*base_cut)[size_t(k)] = std::min(std::max(b, lo), hi);
  }
  return true;
}

namespace {

struct Member {
  int32_t cell;  // tree index
  int32_t slot;  // 2 dir + side
};

}  // namespace

void build_subdomain(const Tree& t, const std::vector<int64_t>& starts,
                     const std::vector<int64_t>& base_cut, int rank, SubDomain* out) {
  const int D = t.dim(), F = 2 * D, S = D == 3 ? 9 : 3;
  const int R = int(base_cut.size()) - 1;
  SubDomain& sd = *out;
  sd.nranks = R;
  sd.rank = rank;
  sd.base_cut = base_cut;
  sd.cut.resize(size_t(R) + 1);
  for (int k = 0; k <= R; ++k) sd.cut[size_t(k)] = starts[size_t(base_cut[size_t(k)])];
  const int64_t g0 = sd.cut[size_t(rank)], g1 = sd.cut[size_t(rank) + 1];
  const int64_t nown = g1 - g0;
  sd.first = g0;
  auto owner = [&](int64_t g) {
    return int(std::upper_bound(sd.cut.begin(), sd.cut.end(), g) - sd.cut.begin()) - 1;
  };
  auto owned = [&](int64_t g) { return g >= g0 && g < g1; };

  // local faces: every face with an owned cell (conforming faces of the
  // tree's conf_all order, parent families of its parents order)
  std::vector<ConfFace> gconf;
  for (const ConfFace& f : t.conf_all)
    if (owned(f.left) || owned(f.right)) gconf.push_back(f);
  std::vector<int32_t> gpar;
  for (size_t p = 0; p < t.parents.size(); ++p) {
    bool any = owned(t.parents[p].coarse);
    for (int s = 0; s < S && !any; ++s) any = owned(t.child_fine[p * S + size_t(s)]);
    if (any) gpar.push_back(int32_t(p));
  }
  std::vector<int32_t> ghosts;
  for (const ConfFace& f : gconf) {
    if (!owned(f.left)) ghosts.push_back(f.left);
    if (!owned(f.right)) ghosts.push_back(f.right);
  }
  for (int32_t p : gpar) {
    if (!owned(t.parents[size_t(p)].coarse)) ghosts.push_back(t.parents[size_t(p)].coarse);
    for (int s = 0; s < S; ++s) {
      const int32_t fc = t.child_fine[size_t(p) * S + size_t(s)];
      if (!owned(fc)) ghosts.push_back(fc);
    }
  }
  std::sort(ghosts.begin(), ghosts.end());
  ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
  sd.ghosts = ghosts;
  auto local = [&](int64_t g) -> int32_t {
    if (owned(g)) return int32_t(g - g0);
    return int32_t(nown + (std::lower_bound(ghosts.begin(), ghosts.end(), int32_t(g)) - ghosts.begin()));
  };

  // exchange entries (tree cell * F + slot) per peer; a face's members are
  // its cells with the slot each one contributes
  std::vector<std::vector<int64_t>> send(static_cast<size_t>(R)), recv(static_cast<size_t>(R));
  std::vector<Member> mem;
  std::vector<int> owners;
  auto visit = [&]() {
    owners.clear();
    for (const Member& m : mem) owners.push_back(owner(m.cell));
    std::sort(owners.begin(), owners.end());
    owners.erase(std::unique(owners.begin(), owners.end()), owners.end());
    for (const Member& m : mem) {
      const int oc = owner(m.cell);
      const int64_t key = int64_t(m.cell) * F + m.slot;
      if (oc == rank) {
        for (int q : owners)
          if (q != rank) send[size_t(q)].push_back(key);
      } else {
        recv[size_t(oc)].push_back(key);
      }
    }
  };
  for (const ConfFace& f : gconf) {
    mem.assign({{f.left, 2 * f.dir + 1}, {f.right, 2 * f.dir + 0}});
    visit();
  }
  for (int32_t p : gpar) {
    const ParentFace& pf = t.parents[size_t(p)];
    mem.assign({{pf.coarse, 2 * pf.dir + pf.coarse_side}});
    for (int s = 0; s < S; ++s)
      mem.push_back({t.child_fine[size_t(p) * S + size_t(s)], 2 * pf.dir + (1 - pf.coarse_side)});
    visit();
  }
  sd.send.assign(size_t(R), {});
  sd.recv.assign(size_t(R), {});
  std::vector<uint8_t> sent(size_t(nown), 0);
  for (int q = 0; q < R; ++q) {
    for (auto* lists : {&send, &recv}) {
      std::vector<int64_t>& v = (*lists)[size_t(q)];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      std::vector<int32_t>& dst = lists == &send ? sd.send[size_t(q)] : sd.recv[size_t(q)];
      dst.reserve(v.size());
      for (int64_t key : v) {
        const int64_t g = key / F;
        dst.push_back(int32_t(int64_t(local(g)) * F + key % F));
        if (lists == &send) sent[size_t(g - g0)] = 1;
      }
    }
  }

  // local lists
  MeshLists& L = sd.lists;
  L = MeshLists();
  L.nowned = nown;
  L.nlocal = nown + int64_t(ghosts.size());
  L.levels.resize(size_t(L.nlocal));
  for (int64_t i = 0; i < nown; ++i) L.levels[size_t(i)] = int8_t(t.cells[size_t(g0 + i)].level);
  for (size_t g = 0; g < ghosts.size(); ++g)
    L.levels[size_t(nown) + g] = int8_t(t.cells[size_t(ghosts[g])].level);
  std::vector<uint8_t> skel(size_t(nown), 0);
  for (int64_t i = 0; i < nown; ++i) {
    skel[size_t(i)] = t.skeleton[size_t(g0 + i)] || sent[size_t(i)];
    (skel[size_t(i)] ? L.skel_cells : L.encl_cells).push_back(int32_t(i));
  }
  std::vector<ConfFace> rest;
  for (const ConfFace& f : gconf) {
    const ConfFace lf{local(f.left), local(f.right), f.dir, 0};
    const bool both = lf.left < nown && lf.right < nown && skel[size_t(lf.left)] && skel[size_t(lf.right)];
    (both ? L.conf : rest).push_back(lf);
  }
  L.n_conf_skeleton = int64_t(L.conf.size());
  L.conf.insert(L.conf.end(), rest.begin(), rest.end());
  for (int32_t p : gpar) {
    const ParentFace& pf = t.parents[size_t(p)];
    L.parents.push_back({local(pf.coarse), pf.dir, pf.coarse_side, 0});
    for (int s = 0; s < S; ++s) L.child_fine.push_back(local(t.child_fine[size_t(p) * S + size_t(s)]));
  }
  // no enclave pipeline in a sub-domain: one chunk, every cell corrected last
  L.chunks = 1;
  L.chunk_off = {0, int64_t(L.encl_cells.size())};
  L.face_off = {0, int64_t(L.conf.size()) - L.n_conf_skeleton};
  L.corr_off = {0, 0, nown};
  L.corr_cells.resize(size_t(nown));
  for (int64_t i = 0; i < nown; ++i) L.corr_cells[size_t(i)] = int32_t(i);
}

}  // namespace ader
