// Octree and interaction lists (host, setup only).
//
// Sec. II-C applies the FMM to the panels in "particle simulation format"
// (panel centroids as particles); the tree below is this library's design:
//  - root cube: lo = component-wise minimum of the centroids, side = largest
//    extent * (1 + 2^-20); centroid c -> integer cell q = floor((c - lo) / side
//    * 2^21) clamped to 2^21 - 1; 63-bit Morton key with x in bit 3b, y in
//    3b + 1, z in 3b + 2 (computed on the GPU, see geom.cu);
//  - panels sorted by (key, caller index);
//  - uniform depth: the leaf level L is the smallest level >= 2 at which the
//    mean occupancy of the non-empty boxes is <= leaf_target (at most 20),
//    and never above level 2;
//  - only non-empty boxes exist; a box's children are the non-empty boxes of
//    the next level with its key as prefix;
//  - every list is sorted by box index (= Morton order within a level);
//    distinct (target - source) V-list cell offsets are numbered in
//    lexicographic (dx, dy, dz) order.
// Two rules decide which pairs of boxes are far enough apart for the
// translated expansions:
//  - bounding spheres (mac_theta > 0): box centre c_b = lo + (cell + 1/2) h_l,
//    radius rho_b = largest distance from c_b to a vertex of a panel in the
//    box (panels may stick out of their box; their surfaces lie within
//    rho_b); boxes t, s of one level are well separated when
//    rho_t + rho_s <= mac_theta |c_t - c_s|.  Every level-1 pair is near; at
//    level l >= 2 the candidates of t are the children of the near boxes of
//    t's parent, split into t's V-list (well separated) and its near list;
//    the leaf level's near lists are the U-lists.  Distances are summed
//    x, y, z in that order (host code is built without FMA contraction) so
//    that a second implementation of the same rule can agree bit for bit;
//  - cell distance (mac_theta = 0, separation ws = 1 or 2): two boxes of one
//    level are NEIGHBOURS when their cells differ by at most ws in every
//    direction; U-list of a leaf: non-empty neighbouring leaves (itself
//    included); V-list of a box at level >= 2: non-empty children of the
//    parent's neighbours (the parent included) that are not neighbours of
//    the box.  This rule also caps the depth so that leaf sides are >= 2 r_max
//    (r_max = largest centroid-to-vertex distance), since it cannot see
//    panels that stick out of their boxes.
// Either way every panel pair is covered exactly once: by the U-list of its
// leaf pair, or by the V-list pair at the unique level where its two
// ancestors first count as well separated.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "xrl_internal.hpp"

namespace xrl {

uint64_t morton_key(uint32_t ix, uint32_t iy, uint32_t iz) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= (uint64_t)((ix >> b) & 1u) << (3 * b);
    k |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);
    k |= (uint64_t)((iz >> b) & 1u) << (3 * b + 2);
  }
  return k;
}

void morton_decode(uint64_t key, uint32_t* ix, uint32_t* iy, uint32_t* iz) {
  uint32_t x = 0, y = 0, z = 0;
  for (int b = 0; b < 21; ++b) {
    x |= (uint32_t)((key >> (3 * b)) & 1u) << b;
    y |= (uint32_t)((key >> (3 * b + 1)) & 1u) << b;
    z |= (uint32_t)((key >> (3 * b + 2)) & 1u) << b;
  }
  *ix = x;
  *iy = y;
  *iz = z;
}

namespace {

int64_t find_key(const std::vector<uint64_t>& keys, int64_t lo, int64_t hi, uint64_t k) {
  auto b = keys.begin() + lo, e = keys.begin() + hi;
  auto it = std::lower_bound(b, e, k);
  if (it != e && *it == k) return it - keys.begin();
  return -1;
}

// Interaction lists by the bounding-sphere rule (see the file header).
void mac_lists(xrl_ctx* c, const std::vector<uint64_t>& sk, const std::vector<std::vector<int32_t>>& first_of,
               double theta) {
  Tree& t = c->tree;
  const int L = t.L, N = (int)sk.size(), nb = t.n_boxes();
  // box centres and radii
  std::vector<double> ctr(3 * (size_t)nb), rad(nb, 0.0);
  std::vector<int32_t> cell(3 * (size_t)nb);
  for (int l = 0; l <= L; ++l) {
    const double h = t.side / (double)(1u << l);
    const int b0 = t.level_off[l], nbl = t.level_off[l + 1] - b0;
    for (int i = 0; i < nbl; ++i) {
      const int b = b0 + i;
      uint32_t x, y, z;
      morton_decode(t.box_key[b], &x, &y, &z);
      cell[3 * (size_t)b] = (int32_t)x;
      cell[3 * (size_t)b + 1] = (int32_t)y;
      cell[3 * (size_t)b + 2] = (int32_t)z;
      const double cc[3] = {t.lo[0] + ((double)x + 0.5) * h, t.lo[1] + ((double)y + 0.5) * h,
                            t.lo[2] + ((double)z + 0.5) * h};
      for (int k = 0; k < 3; ++k) ctr[3 * (size_t)b + k] = cc[k];
      const int r0 = first_of[l][i], r1 = (i + 1 < nbl) ? first_of[l][i + 1] : N;
      double r2 = 0.0;
      for (int r = r0; r < r1; ++r) {
        const int p = t.perm[r];
        for (int v = 0; v < panel_nv(c->pan, p); ++v) {
          const double* X = &c->xyz[3 * (size_t)c->pan[4 * (size_t)p + v]];
          const double dx = X[0] - cc[0], dy = X[1] - cc[1], dz = X[2] - cc[2];
          const double d2 = dx * dx + dy * dy + dz * dz;
          if (d2 > r2) r2 = d2;
        }
      }
      rad[b] = std::sqrt(r2);
    }
  }
  // children of a box are contiguous at the next level
  std::vector<int32_t> cfirst(nb, 0), clast(nb, 0);
  for (int b = t.level_off[1]; b < nb; ++b) {
    const int P = t.parent[b];
    if (clast[P] == 0) cfirst[P] = b;
    clast[P] = b + 1;
  }
  auto separated = [&](int a, int b) {
    const double dx = ctr[3 * (size_t)a] - ctr[3 * (size_t)b];
    const double dy = ctr[3 * (size_t)a + 1] - ctr[3 * (size_t)b + 1];
    const double dz = ctr[3 * (size_t)a + 2] - ctr[3 * (size_t)b + 2];
    const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
    return a != b && rad[a] + rad[b] <= theta * dist;
  };
  // near lists of the current level (global ids), starting with level 1: all pairs
  std::vector<int64_t> nptr{0};
  std::vector<int32_t> nsrc;
  {
    const int b0 = t.level_off[1], b1 = t.level_off[2];
    for (int a = b0; a < b1; ++a) {
      for (int b = b0; b < b1; ++b) nsrc.push_back(b);
      nptr.push_back((int64_t)nsrc.size());
    }
  }
  t.v_ptr.assign(nb + 1, 0);
  t.v_src.clear();
  std::vector<int64_t> vcode;
  const int64_t K = 1 << 20;
  auto code_of = [&](int tg, int sc) {
    const int64_t dx = cell[3 * (size_t)tg] - cell[3 * (size_t)sc], dy = cell[3 * (size_t)tg + 1] - cell[3 * (size_t)sc + 1],
                  dz = cell[3 * (size_t)tg + 2] - cell[3 * (size_t)sc + 2];
    return ((dx + K) << 42) | ((dy + K) << 21) | (dz + K);
  };
  for (int l = 2; l <= L; ++l) {
    const int b0 = t.level_off[l], b1 = t.level_off[l + 1], pb0 = t.level_off[l - 1];
    std::vector<int64_t> mptr{0};
    std::vector<int32_t> msrc;
    for (int tg = b0; tg < b1; ++tg) {
      const int P = t.parent[tg] - pb0;
      std::vector<int32_t> vl, nl;
      for (int64_t k = nptr[P]; k < nptr[P + 1]; ++k) {
        const int sp = nsrc[k];
        for (int sc = cfirst[sp]; sc < clast[sp]; ++sc) (separated(tg, sc) ? vl : nl).push_back(sc);
      }
      std::sort(vl.begin(), vl.end());
      std::sort(nl.begin(), nl.end());
      for (int sc : vl) {
        t.v_src.push_back(sc);
        vcode.push_back(code_of(tg, sc));
      }
      t.v_ptr[tg + 1] = (int64_t)t.v_src.size();
      msrc.insert(msrc.end(), nl.begin(), nl.end());
      mptr.push_back((int64_t)msrc.size());
    }
    nptr.swap(mptr);
    nsrc.swap(msrc);
  }
  // boxes of levels 0, 1 have empty V-lists: carry the pointer forward
  for (int b = 0; b < nb; ++b) t.v_ptr[b + 1] = std::max(t.v_ptr[b + 1], t.v_ptr[b]);
  // U-lists: the leaf level's near lists, leaf-local
  const int leaf0 = t.level_off[L], nl = t.n_leaves();
  t.u_ptr.assign(nl + 1, 0);
  t.u_src.clear();
  for (int i = 0; i < nl; ++i) {
    for (int64_t k = nptr[i]; k < nptr[i + 1]; ++k) t.u_src.push_back(nsrc[k] - leaf0);
    t.u_ptr[i + 1] = (int64_t)t.u_src.size();
  }
  // compact offset table
  std::vector<int64_t> used(vcode);
  std::sort(used.begin(), used.end());
  used.erase(std::unique(used.begin(), used.end()), used.end());
  XRL_CHECK(used.size() < 32768, XRL_EINVAL, "too many M2L offsets");
  t.m2l_offsets.clear();
  for (int64_t code : used) {
    const int dz = (int)((code & ((1 << 21) - 1)) - K), dy = (int)(((code >> 21) & ((1 << 21) - 1)) - K),
              dx = (int)((code >> 42) - K);
    t.m2l_offsets.insert(t.m2l_offsets.end(), {dx, dy, dz});
  }
  t.v_off.resize(vcode.size());
  for (size_t k = 0; k < vcode.size(); ++k)
    t.v_off[k] = (int16_t)(std::lower_bound(used.begin(), used.end(), vcode[k]) - used.begin());
}

}  // namespace

void build_tree(xrl_ctx* c, const std::vector<uint64_t>& keys) {
  Tree& t = c->tree;
  const int N = (int)keys.size();
  t.key = keys;
  t.perm.resize(N);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  std::stable_sort(t.perm.begin(), t.perm.end(), [&](int a, int b) { return keys[a] < keys[b]; });
  t.rank.assign(N, 0);
  for (int r = 0; r < N; ++r) t.rank[t.perm[r]] = r;
  std::vector<uint64_t> sk(N);
  for (int r = 0; r < N; ++r) sk[r] = keys[t.perm[r]];

  const int target = std::max(1, c->opt.leaf_target);
  int L = 20;
  for (int l = 2; l <= 20; ++l) {
    int shift = 3 * (21 - l);
    int64_t cnt = 0;
    for (int r = 0; r < N; ++r)
      if (r == 0 || (sk[r] >> shift) != (sk[r - 1] >> shift)) ++cnt;
    if ((double)N / (double)cnt <= (double)target) {
      L = l;
      break;
    }
  }
  // size cap: side / 2^l >= 2 r_max
  double rmax = 0.0;
  for (int p = 0; p < N; ++p) {
    const int32_t* tv = &c->pan[4 * (size_t)p];
    double cc[3];
    panel_centroid_host(c->xyz, c->pan, p, cc);
    for (int v = 0; v < panel_nv(c->pan, p); ++v) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        double d = c->xyz[3 * (size_t)tv[v] + k] - cc[k];
        d2 += d * d;
      }
      rmax = std::max(rmax, std::sqrt(d2));
    }
  }
  int Lsize = 2;
  for (int l = 2; l <= 20; ++l)
    if (t.side / (double)(1 << l) >= 2.0 * rmax) Lsize = l;
  const double theta = c->opt.mac_theta;
  t.L = theta > 0 ? std::max(2, L) : std::max(2, std::min(L, Lsize));
  L = t.L;

  // boxes per level
  t.level_off.assign(L + 2, 0);
  t.box_key.clear();
  std::vector<std::vector<int32_t>> first_of(L + 1);
  for (int l = 0; l <= L; ++l) {
    t.level_off[l] = (int)t.box_key.size();
    int shift = 3 * (21 - l);
    for (int r = 0; r < N; ++r)
      if (r == 0 || (sk[r] >> shift) != (sk[r - 1] >> shift)) {
        t.box_key.push_back(sk[r] >> shift);
        first_of[l].push_back(r);
      }
  }
  t.level_off[L + 1] = (int)t.box_key.size();
  const int nb = (int)t.box_key.size();
  t.parent.assign(nb, -1);
  t.octant.assign(nb, 0);
  for (int l = 1; l <= L; ++l)
    for (int b = t.level_off[l]; b < t.level_off[l + 1]; ++b) {
      uint64_t pk = t.box_key[b] >> 3;
      int64_t pb = find_key(t.box_key, t.level_off[l - 1], t.level_off[l], pk);
      XRL_CHECK(pb >= 0, XRL_EINVAL, "tree: missing parent");
      t.parent[b] = (int)pb;
      t.octant[b] = (int)(t.box_key[b] & 7u);
    }
  // leaves
  const int nl = t.level_off[L + 1] - t.level_off[L];
  t.leaf_first.assign(nl, 0);
  t.leaf_count.assign(nl, 0);
  t.leaf_of.assign(N, 0);
  for (int i = 0; i < nl; ++i) {
    t.leaf_first[i] = first_of[L][i];
    int end = (i + 1 < nl) ? first_of[L][i + 1] : N;
    t.leaf_count[i] = end - t.leaf_first[i];
    for (int r = t.leaf_first[i]; r < end; ++r) t.leaf_of[r] = i;
  }
  if (theta > 0) {
    mac_lists(c, sk, first_of, theta);
    return;
  }
  const int ws = c->opt.separation;
  // U-lists
  t.u_ptr.assign(nl + 1, 0);
  t.u_src.clear();
  for (int i = 0; i < nl; ++i) {
    uint32_t x, y, z;
    morton_decode(t.box_key[t.level_off[L] + i], &x, &y, &z);
    std::vector<int32_t> lst;
    const int64_t lim = (int64_t)1 << L;
    for (int dx = -ws; dx <= ws; ++dx)
      for (int dy = -ws; dy <= ws; ++dy)
        for (int dz = -ws; dz <= ws; ++dz) {
          int64_t X = (int64_t)x + dx, Y = (int64_t)y + dy, Z = (int64_t)z + dz;
          if (X < 0 || Y < 0 || Z < 0 || X >= lim || Y >= lim || Z >= lim) continue;
          int64_t g = find_key(t.box_key, t.level_off[L], t.level_off[L + 1],
                               morton_key((uint32_t)X, (uint32_t)Y, (uint32_t)Z));
          if (g >= 0) lst.push_back((int32_t)(g - t.level_off[L]));
        }
    std::sort(lst.begin(), lst.end());
    t.u_src.insert(t.u_src.end(), lst.begin(), lst.end());
    t.u_ptr[i + 1] = (int64_t)t.u_src.size();
  }
  // V-lists (levels >= 2); offsets first collected as full codes
  const int R = 2 * ws + 1, D = 2 * R + 1;
  t.v_ptr.assign(nb + 1, 0);
  t.v_src.clear();
  t.v_off.clear();
  std::vector<int32_t> full_code;
  for (int b = 0; b < nb; ++b) {
    int l = 0;
    while (b >= t.level_off[l + 1]) ++l;
    std::vector<std::pair<int32_t, int32_t>> lst;
    if (l >= 2) {
      uint32_t x, y, z;
      morton_decode(t.box_key[b], &x, &y, &z);
      uint32_t px = x >> 1, py = y >> 1, pz = z >> 1;
      const int64_t plim = (int64_t)1 << (l - 1);
      for (int dx = -ws; dx <= ws; ++dx)
        for (int dy = -ws; dy <= ws; ++dy)
          for (int dz = -ws; dz <= ws; ++dz) {
            int64_t X = (int64_t)px + dx, Y = (int64_t)py + dy, Z = (int64_t)pz + dz;
            if (X < 0 || Y < 0 || Z < 0 || X >= plim || Y >= plim || Z >= plim) continue;
            uint64_t nk = morton_key((uint32_t)X, (uint32_t)Y, (uint32_t)Z);
            if (find_key(t.box_key, t.level_off[l - 1], t.level_off[l], nk) < 0) continue;
            for (int o = 0; o < 8; ++o) {
              uint64_t ck = (nk << 3) | (uint64_t)o;
              int64_t g = find_key(t.box_key, t.level_off[l], t.level_off[l + 1], ck);
              if (g < 0) continue;
              uint32_t cx, cy, cz;
              morton_decode(ck, &cx, &cy, &cz);
              int ddx = (int)cx - (int)x, ddy = (int)cy - (int)y, ddz = (int)cz - (int)z;
              if (std::max(std::abs(ddx), std::max(std::abs(ddy), std::abs(ddz))) <= ws) continue;
              // full code of the (target - source) offset in box units
              int32_t code = ((-ddx + R) * D + (-ddy + R)) * D + (-ddz + R);
              lst.push_back({(int32_t)g, code});
            }
          }
      std::sort(lst.begin(), lst.end());
    }
    for (auto& pr : lst) {
      t.v_src.push_back(pr.first);
      full_code.push_back(pr.second);
    }
    t.v_ptr[b + 1] = (int64_t)t.v_src.size();
  }
  // compact offset table: distinct codes in increasing order
  std::vector<int32_t> used(full_code);
  std::sort(used.begin(), used.end());
  used.erase(std::unique(used.begin(), used.end()), used.end());
  XRL_CHECK(used.size() < 32768, XRL_EINVAL, "too many M2L offsets");
  t.m2l_offsets.clear();
  for (int32_t code : used) {
    int dz = code % D - R, dy = (code / D) % D - R, dx = code / (D * D) - R;
    t.m2l_offsets.insert(t.m2l_offsets.end(), {dx, dy, dz});
  }
  t.v_off.resize(full_code.size());
  for (size_t k = 0; k < full_code.size(); ++k)
    t.v_off[k] = (int16_t)(std::lower_bound(used.begin(), used.end(), full_code[k]) - used.begin());
}

}  // namespace xrl
