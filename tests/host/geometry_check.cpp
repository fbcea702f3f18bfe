// Host-side checks of the mirrored-pair bookkeeping in vet_geometry.h (no GPU):
//  - mirror_octant_order puts antipodes at equal positions of opposite octants;
//  - the cell- and node-ray parts of each antipodal pair's templates are
//    exact mirrors (rotated sets), and a template is not the mirror of a
//    direction other than its antipode;
//  - the paired cell pass marches every antipodal pair of a rotated set as a
//    mirrored pair, and never one with a zero direction component (whose
//    sign the antipode keeps) of the unrotated set;
//  - the paired face pass's node orders (per template: each face axis, and
//    the three faces merged) are permutations of the nodes within 31
//    places of their order by node-ray length;
//  - the paired face-pass schedule, with each item's point-mirrored block and
//    antipodal directions added, lists every (block, direction) of the
//    unpaired schedule exactly once, level by level.
// Usage: geometry_check nbx nby nbz B nside [unrotated]   (prints "ok" or the
// failure).  The rotation is a generic one (irrational components: no two
// plane crossings of a direction tie); "unrotated" checks instead that the
// HEALPix set itself, with its z = 0 ring, is refused by the face pass's
// mirror order and its zero-component pairs by the cell pass's pairing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <tuple>
#include <vector>

#include "vet_geometry.h"

static int fail(const char *what) {
  std::printf("FAIL: %s\n", what);
  return 1;
}

int main(int argc, char **argv) {
  if (argc != 6 && argc != 7) return fail("usage");
  const int nb[3] = {std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3])};
  const int B = std::atoi(argv[4]), nside = std::atoi(argv[5]), N = 12 * nside * nside;
  const bool unrotated = argc == 7;
  double q[4] = {std::sqrt(0.5), 1.0 / std::sqrt(10.0), 1.0 / std::sqrt(3.0), 0.2};
  if (unrotated) q[0] = 1.0, q[1] = q[2] = q[3] = 0.0;
  const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (double &x : q) x /= qn;
  std::vector<double> d(4 * N);
  vet::geom::healpix_directions(nside, q, d.data());
  std::vector<int> order(N);
  int ob[9];
  vet::geom::internal_order(N, d.data(), order.data(), ob);
  const int tb = vet::tpl_layout<float>(B).bytes;
  std::vector<unsigned char> tpl((size_t)tb * N);
  auto T = [&](int i) { return tpl.data() + (size_t)i * tb; };
  auto build_templates = [&]() {
    for (int i = 0; i < N; ++i) {
      long long cs, ns[3];
      vet::geom::build_template<float>(&d[4 * order[i]], order[i], B, 0.01, T(i), cs, ns);
    }
  };
  // the paired cell pass: pairs (cell_order[2k], cell_order[2k + 1]) of antipodes
  auto check_cell_pairs = [&](bool rotated) -> int {
    std::vector<int> cell_order(N);
    vet::geom::interleaved_order(ob, cell_order.data());
    if (!vet::geom::antipodal_order(N, d.data(), order.data(), cell_order.data()))
      return fail("antipodal_order refused a set closed under negation");
    int zero_pairs = 0;
    for (int k = 0; k < N; k += 2) {
      const int i = cell_order[k], j = cell_order[k + 1];
      const double *a = &d[4 * order[i]];
      const bool zero = a[0] == 0.0 || a[1] == 0.0 || a[2] == 0.0;
      const bool m = vet::geom::mirrored_cell_pair<float>(T(i), T(j), B);
      if (zero && m) return fail("a pair with a zero direction component was marked mirrored");
      if (rotated && !m) return fail("an antipodal pair of a rotated set was not marked mirrored");
      zero_pairs += zero ? 1 : 0;
    }
    if (!rotated && zero_pairs == 0) return fail("the unrotated set has no zero component to check");
    return 0;
  };
  if (unrotated) {
    const std::vector<int> before = order;
    if (vet::geom::mirror_octant_order(N, d.data(), order.data(), ob)) return fail("a set with zero components was paired");
    if (order != before) return fail("a refused mirror order changed the order");
    build_templates();
    if (check_cell_pairs(false)) return 1;
    std::printf("ok\n");
    return 0;
  }
  if (!vet::geom::mirror_octant_order(N, d.data(), order.data(), ob)) return fail("mirror_octant_order refused a rotated set");
  for (int o = 0; o < 8; o += 2)
    for (int k = 0; k < ob[o + 1] - ob[o]; ++k) {
      const double *a = &d[4 * order[ob[o] + k]], *b = &d[4 * order[ob[7 - o] + k]];
      if (std::fabs(a[0] + b[0]) + std::fabs(a[1] + b[1]) + std::fabs(a[2] + b[2]) > 1e-12)
        return fail("octant positions do not hold antipodes");
    }
  build_templates();
  if (check_cell_pairs(true)) return 1;
  for (int o = 0; o < 8; o += 2)
    for (int k = 0; k < ob[o + 1] - ob[o]; ++k) {
      const int i = ob[o] + k, j = ob[7 - o] + k;
      if (!vet::geom::mirror_node_templates<float>(T(i), T(j), B)) return fail("node rays of an antipodal pair");
      if (!vet::geom::mirror_templates<float>(T(i), T(j), B)) return fail("cell rays of an antipodal pair");
      const int other = ob[7 - o] + (k + 1) % (ob[o + 1] - ob[o]);
      if (other != j && vet::geom::mirror_node_templates<float>(T(i), T(other), B))
        return fail("a non-antipodal pair passed the node mirror check");
    }
  // the paired face pass's node order: per template, for each face axis a
  // permutation of the (B+1)^2 face nodes, then one of the codes of all
  // three faces, each node within 31 places of its rank by the node ray's
  // exit parameter min_b L_b / |n_b| (L: the node's upwind-frame
  // coordinates, B along the face's axis; the ray leaves the block where
  // the first of them reaches 0)
  {
    const int N1 = B + 1, NN = N1 * N1;
    std::vector<uint16_t> no((size_t)6 * NN);
    for (int i = 0; i < N; ++i) {
      vet::geom::node_order<float>(T(i), B, no.data());
      const double *dir = &d[4 * order[i]];
      auto exit_t = [&](int code) {
        const int a = code / NN, r = code % NN, ub = r / N1, uc = r % N1;
        const int L[3] = {a == 0 ? B : ub, a == 1 ? B : (a == 0 ? ub : uc), a == 2 ? B : uc};
        double t = 1e300;
        for (int b = 0; b < 3; ++b) t = std::min(t, L[b] / std::fabs(dir[b]));
        return t;
      };
      // (first code, count, offset of the list in no, value offset)
      for (int part = 0; part < 4; ++part) {
        const int c0 = part < 3 ? part * NN : 0, n = part < 3 ? NN : 3 * NN;
        const uint16_t *o = no.data() + (part < 3 ? part * NN : 3 * NN);
        std::vector<double> ts(n);
        for (int k = 0; k < n; ++k) ts[k] = exit_t(c0 + k);
        std::sort(ts.begin(), ts.end());
        std::vector<int> seen(n, 0);
        for (int k = 0; k < n; ++k) {
          const int code = o[k] + (part < 3 ? c0 : 0);
          if (code - c0 < 0 || code - c0 >= n || seen[code - c0]++)
            return fail("node order is not a permutation of a face's nodes");
          const double t = exit_t(code);
          if (t < ts[std::max(0, k - 31)] - 1e-9 || t > ts[std::min(n - 1, k + 31)] + 1e-9)
            return fail("node order is not by ray length");
        }
      }
    }
  }
  const int nl = nb[0] + nb[1] + nb[2] - 2;
  for (int g : {1, 2, 4, 8}) {
    std::vector<int> off(nl + 1), poff(nl + 1);
    const long long nu = vet::geom::build_schedule(nb, ob, g, nullptr, 1LL << 40, off.data());
    std::vector<vet::FaceItem> U((size_t)nu + 1);
    vet::geom::build_schedule(nb, ob, g, U.data(), nu, off.data());
    const long long np = vet::geom::build_schedule(nb, ob, g, nullptr, 1LL << 40, poff.data(), nullptr, true);
    std::vector<vet::FaceItem> P((size_t)np + 1);
    vet::geom::build_schedule(nb, ob, g, P.data(), np, poff.data(), nullptr, true);
    for (int L = 0; L < nl; ++L) {
      std::multiset<std::tuple<int, int>> a, b;
      for (int i = off[L]; i < off[L + 1]; ++i)
        for (int j = 0; j < U[i].dir_count; ++j) {
          a.insert({U[i].block, U[i].dir_begin + j});
          if (vet::geom::octant_of(&d[4 * order[U[i].dir_begin + j]]) != U[i].octant)
            return fail("item octant differs from its directions'");
        }
      for (int i = poff[L]; i < poff[L + 1]; ++i) {
        const int bx = P[i].block % nb[0], by = (P[i].block / nb[0]) % nb[1], bz = P[i].block / (nb[0] * nb[1]);
        const int mb = ((nb[2] - 1 - bz) * nb[1] + (nb[1] - 1 - by)) * nb[0] + (nb[0] - 1 - bx);
        if (P[i].dir_count > g) return fail("paired item larger than its group");
        for (int j = 0; j < P[i].dir_count; ++j) {
          b.insert({P[i].block, P[i].dir_begin + j});
          b.insert({mb, P[i].mirror_begin + j});
          const double *x = &d[4 * order[P[i].dir_begin + j]], *y = &d[4 * order[P[i].mirror_begin + j]];
          if (vet::geom::octant_of(x) != P[i].octant || vet::geom::octant_of(y) != 7 - P[i].octant)
            return fail("paired item octant differs from its directions'");
          if (std::fabs(x[0] + y[0]) + std::fabs(x[1] + y[1]) + std::fabs(x[2] + y[2]) > 1e-12)
            return fail("paired item's mirror directions are not antipodes");
        }
      }
      if (a != b) return fail("paired schedule does not cover the unpaired one");
    }
    if (2 * np != nu) return fail("paired schedule is not half the unpaired one");
  }
  std::printf("ok\n");
  return 0;
}
