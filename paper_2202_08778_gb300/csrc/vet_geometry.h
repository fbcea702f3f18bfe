// vet_geometry.h -- host-side geometry of the VET closure, shared by the
// context path (vet_host.cu) and the allocation-free path (vet_noalloc.cu):
// the HEALPix direction set, the per-direction ray templates, the internal
// direction orders and the wavefront schedule of the face pass.  Every
// function writes into caller-provided memory and allocates nothing.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "vet_internal.h"

namespace vet {
namespace geom {

// HEALPix ring-scheme pixel centres (Gorski et al. 2005, Sec. 4): north cap
// rings i < nside at z = 1 - i^2/(3 nside^2) with 4i pixels at
// phi = (j - 1/2) pi/(2i); equatorial rings nside <= i <= 3 nside at
// z = 4/3 - 2i/(3 nside) with 4 nside pixels at phi = (j - s/2) pi/(2 nside),
// s = (i - nside + 1) mod 2; south cap mirrored.  Then rotated by the unit
// quaternion q (the paper's random rotation, Sec. 2.2.5).  out: [N][4] =
// (nx, ny, nz, w) with w = 4 pi / N.
inline void healpix_directions(int nside, const double q_in[4], double *out) {
  const double pi = 3.14159265358979323846;
  const int N = 12 * nside * nside;
  const double qn = std::sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  const double qw = q_in[0] / qn, qx = q_in[1] / qn, qy = q_in[2] / qn, qz = q_in[3] / qn;
  const double R[3][3] = {
      {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
      {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
      {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
  int p = 0;
  for (int ring = 1; ring < 4 * nside; ++ring) {
    int cnt;
    double z, first, step;
    if (ring < nside || ring > 3 * nside) {
      const int i = ring < nside ? ring : 4 * nside - ring;
      const double zz = 1.0 - double(i) * i / (3.0 * nside * nside);
      z = ring < nside ? zz : -zz;
      cnt = 4 * i;
      step = pi / (2.0 * i);
      first = 0.5 * step;
    } else {
      z = 4.0 / 3.0 - 2.0 * ring / (3.0 * nside);
      const int s = (ring - nside + 1) % 2;
      cnt = 4 * nside;
      step = pi / (2.0 * nside);
      first = step * (1.0 - 0.5 * s);
    }
    const double sin_t = std::sqrt((1.0 - z) * (1.0 + z));
    for (int j = 0; j < cnt; ++j, ++p) {
      const double phi = first + j * step;
      const double v[3] = {sin_t * std::cos(phi), sin_t * std::sin(phi), z};
      for (int a = 0; a < 3; ++a) out[4 * p + a] = R[a][0] * v[0] + R[a][1] * v[1] + R[a][2] * v[2];
      out[4 * p + 3] = 4.0 * pi / N;
    }
  }
}

struct Event {
  double t;
  int axis, m;
};

// Merge order of plane crossings: by parameter, ties to the lowest axis (no
// two events share both, so the order is total).
inline void merge_events(Event *ev, int n) {
  std::sort(ev, ev + n, [](const Event &a, const Event &b) { return a.t < b.t || (a.t == b.t && a.axis < b.axis); });
}

// Ray templates of one direction for block edge B (cell units; segment
// lengths are stored as -length * h * log2(e)), written into the blob `out`
// laid out by tpl_layout.  Returns in cell_segs / node_segs the segments a
// block's cell rays and face-node rays cross for this direction.
template <typename R>
void build_template(const double *d, int ext, int B, double h, unsigned char *out, long long &cell_segs,
                    long long node_segs[3]) {
  const TplLayout L = tpl_layout<R>(B);
  std::memset(out, 0, L.bytes);
  auto *hd = reinterpret_cast<TplHead<R> *>(out);
  auto *cev = reinterpret_cast<TplEvent<R> *>(out + L.cev);
  auto *nev = reinterpret_cast<TplEvent<R> *>(out + L.nev);
  int16_t *cpos = reinterpret_cast<int16_t *>(out + L.cpos);
  int16_t *npos = reinterpret_cast<int16_t *>(out + L.npos);
  int16_t *ck = reinterpret_cast<int16_t *>(out + L.ck);
  R *cw = reinterpret_cast<R *>(out + L.cw);
  int16_t *nk = reinterpret_cast<int16_t *>(out + L.nk);
  R *nw = reinterpret_cast<R *>(out + L.nw);
  const double scale = -h * 1.4426950408889634074;  // -h log2(e)
  double an[3];
  int sgn[3];
  for (int a = 0; a < 3; ++a) {
    hd->n[a] = R(d[a]);
    an[a] = std::fabs(d[a]);
    sgn[a] = d[a] < 0.0 ? -1 : 1;
    hd->sgn[a] = sgn[a];
  }
  hd->w = R(d[3]);
  hd->ext = ext;
  {
    const double w = d[3], x = d[0], y = d[1], z = d[2];
    const double c[10] = {w, w * x, w * y, w * z, w * x * x, w * y * y, w * z * z, w * x * y, w * x * z, w * y * z};
    for (int m = 0; m < 10; ++m) {
      hd->c[m] = R(c[m]);
      hd->cp[2 * m] = R(c[m]);
      hd->cp[2 * m + 1] = (m >= 1 && m <= 3) ? R(-c[m]) : R(c[m]);
    }
  }
  const TileShape ct = cell_tile(B), nt = node_tile(B);
  const int cstride[3] = {1, ct.sy, ct.sz};  // cell rays walk the cell-pass tile
  const int nstride[3] = {1, nt.sy, nt.sz};  // node rays walk the face-pass tile
  Event ev[3 * kMaxBlock];
  // cell rays: planes at t = (m + 1/2)/|n_a|, m = 0..B-1
  int n = 0;
  for (int a = 0; a < 3; ++a)
    if (an[a] > 0.0)
      for (int m = 0; m < B; ++m) ev[n++] = {(m + 0.5) / an[a], a, m};
  merge_events(ev, n);
  for (int i = 0; i < 3 * B; ++i) cpos[i] = kNever;
  double prev = 0.0;
  int off = 0;
  for (int e = 0; e < n; ++e) {
    cpos[ev[e].axis * B + ev[e].m] = (int16_t)e;
    cev[e].len = R((ev[e].t - prev) * scale);
    cev[e].off = off * (int)(2 * sizeof(R));  // bytes: one (kappa, S) pair per tile cell
    off -= sgn[ev[e].axis] * cstride[ev[e].axis];  // crossing the plane moves one cell upwind
    prev = ev[e].t;
  }
  // node rays: planes at t = m/|n_a|, m = 1..B
  n = 0;
  for (int a = 0; a < 3; ++a)
    if (an[a] > 0.0)
      for (int m = 1; m <= B; ++m) ev[n++] = {m / an[a], a, m};
  merge_events(ev, n);
  for (int a = 0; a < 3; ++a) {
    npos[a * (B + 1)] = -1;
    for (int m = 1; m <= B; ++m) npos[a * (B + 1) + m] = kNever;
  }
  prev = 0.0;
  off = 0;
  for (int e = 0; e < n; ++e) {
    npos[ev[e].axis * (B + 1) + ev[e].m] = (int16_t)e;
    nev[e].len = R((ev[e].t - prev) * scale);
    nev[e].off = off * (int)(2 * sizeof(R));
    off -= sgn[ev[e].axis] * nstride[ev[e].axis];
    prev = ev[e].t;
  }
  // exit tables: leaving through axis a at depth D, the in-plane upwind-frame
  // offset along axis b is d = off - (D / |n_a|) |n_b| (off = 1/2 for cells,
  // 0 for nodes); stored as k = floor(d) and (f, 1 - f), f = d - k.
  auto fill_exit = [&](int16_t *K, R *W, int rows, bool cells) {
    for (int a = 0; a < 3; ++a) {
      const int bc[2] = {a == 0 ? 1 : 0, a == 2 ? 1 : 2};
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < rows; ++l) {
          const int idx = (a * 2 + j) * rows + l;
          double dd = 0.0;
          if (an[a] > 0.0) {
            const double depth = cells ? l + 0.5 : (double)l;
            const double t = depth / an[a];
            dd = (cells ? 0.5 : 0.0) - t * an[bc[j]];
            // an exit exactly on a face edge (a tie with axis b) may come out
            // a rounding error below the integer; snap it so that the device
            // never sees a node index below 0
            const double r = std::nearbyint(dd);
            if (std::fabs(dd - r) < 1e-12) dd = r;
          }
          const double k = std::floor(dd);
          const double f = dd - k;
          K[idx] = (int16_t)k;
          W[2 * idx] = R(f);
          W[2 * idx + 1] = R(1.0 - f);
        }
    }
  };
  fill_exit(ck, cw, B, true);
  fill_exit(nk, nw, B + 1, false);
  // work measure: segments = exit event index + 1 per ray
  long long cs = 0, ns[3] = {0, 0, 0};
  for (int l2 = 0; l2 < B; ++l2)
    for (int l1 = 0; l1 < B; ++l1)
      for (int l0 = 0; l0 < B; ++l0)
        cs += 1 + std::min({(int)cpos[l0], (int)cpos[B + l1], (int)cpos[2 * B + l2]});
  for (int a = 0; a < 3; ++a) {
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    for (int u = 0; u <= B; ++u)
      for (int v = 0; v <= B; ++v) {
        int P[3];
        P[a] = sgn[a] > 0 ? B : 0;
        P[b] = u;
        P[c] = v;
        int Lq[3];
        for (int q = 0; q < 3; ++q) Lq[q] = sgn[q] > 0 ? P[q] : B - P[q];
        ns[a] += 1 + std::min({(int)npos[Lq[0]], (int)npos[(B + 1) + Lq[1]], (int)npos[2 * (B + 1) + Lq[2]]});
      }
  }
  cell_segs = cs;
  for (int a = 0; a < 3; ++a) node_segs[a] = ns[a];
}

inline int octant_of(const double *d) { return (d[0] < 0) + 2 * (d[1] < 0) + 4 * (d[2] < 0); }

// Internal order: octant-major, HEALPix order within an octant.  order[i] is
// the HEALPix index of internal direction i; ob[o]..ob[o+1] the octant ranges.
inline void internal_order(int N, const double *dirs, int *order, int ob[9]) {
  int i = 0;
  for (int o = 0; o < 8; ++o) {
    ob[o] = i;
    for (int k = 0; k < N; ++k)
      if (octant_of(dirs + 4 * k) == o) order[i++] = k;
  }
  ob[8] = i;
}

// Cell-pass visiting order: octants interleaved round robin.
inline void interleaved_order(const int ob[9], int *out) {
  int n = 0;
  for (int r = 0; n < ob[8]; ++r)
    for (int o = 0; o < 8; ++o)
      if (ob[o] + r < ob[o + 1]) out[n++] = ob[o] + r;
}

// Cell order of antipodal pairs: for every internal direction i the
// internal index of -n_i (components equal and opposite within 1e-12), the
// pair listed as (d, -d) with d the member whose first nonzero component is
// positive, pairs in increasing order of d.  Returns false (out untouched)
// when some direction has no antipode in the set.
inline bool antipodal_order(int N, const double *dirs, const int *order, int *out) {
  int *mate = new int[N];
  for (int i = 0; i < N; ++i) mate[i] = -1;
  bool ok = true;
  for (int i = 0; i < N && ok; ++i) {
    if (mate[i] >= 0) continue;
    const double *a = dirs + 4 * order[i];
    for (int j = 0; j < N; ++j) {
      if (j == i || mate[j] >= 0) continue;
      const double *b = dirs + 4 * order[j];
      if (std::fabs(a[0] + b[0]) < 1e-12 && std::fabs(a[1] + b[1]) < 1e-12 && std::fabs(a[2] + b[2]) < 1e-12) {
        mate[i] = j;
        mate[j] = i;
        break;
      }
    }
    ok = mate[i] >= 0;
  }
  if (ok) {
    int n = 0;
    for (int i = 0; i < N; ++i) {
      const double *a = dirs + 4 * order[i];
      const double lead = a[0] != 0.0 ? a[0] : (a[1] != 0.0 ? a[1] : a[2]);
      if (lead > 0.0) {
        out[n++] = i;
        out[n++] = mate[i];
      }
    }
    ok = n == N;
  }
  delete[] mate;
  return ok;
}

// Exit tables of two templates with the same event positions pos[3][rows]:
// equal (floor, fraction within 1e-6) on every row a ray can exit through.
// A ray exits by the plane event that comes first along its three axes, so
// row (a, l) is read only if pos[a][l] is below the latest event of each
// other axis; the other rows (planes the direction would cross only beyond
// the block, as along an axis with a component near zero, whose far-off
// tables differ in rounding between a direction and its antipode) are never
// read.
template <typename R>
inline bool exit_rows_match(const int16_t *pos, const unsigned char *ka, const unsigned char *wa,
                            const unsigned char *kb, const unsigned char *wb, int rows) {
  const int16_t *Ka = reinterpret_cast<const int16_t *>(ka), *Kb = reinterpret_cast<const int16_t *>(kb);
  const R *Wa = reinterpret_cast<const R *>(wa), *Wb = reinterpret_cast<const R *>(wb);
  int latest[3];
  for (int a = 0; a < 3; ++a) {
    latest[a] = pos[a * rows];
    for (int l = 1; l < rows; ++l) latest[a] = std::max(latest[a], (int)pos[a * rows + l]);
  }
  for (int a = 0; a < 3; ++a)
    for (int l = 0; l < rows; ++l) {
      const int p = pos[a * rows + l];
      if (p == kNever || p > latest[(a + 1) % 3] || p > latest[(a + 2) % 3]) continue;
      for (int j = 0; j < 2; ++j) {
        const int idx = (a * 2 + j) * rows + l;
        if (Ka[idx] != Kb[idx]) return false;
        if (std::fabs((double)Wa[2 * idx] - (double)Wb[2 * idx]) > 1e-6) return false;
        if (std::fabs((double)Wa[2 * idx + 1] - (double)Wb[2 * idx + 1]) > 1e-6) return false;
      }
    }
  return true;
}

// Mirrored octant order for the paired face pass: within octant 7 - o (the
// antipodes of octant o, o with a non-negative x component), internal
// direction ob[7 - o] + k becomes the antipode of ob[o] + k.  Requires every
// direction component to be non-zero (so that a direction and its antipode
// lie in opposite octants) and the set to be closed under negation; returns
// false, leaving `order` unchanged, otherwise.
inline bool mirror_octant_order(int N, const double *dirs, int *order, const int ob[9]) {
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a)
      if (dirs[4 * i + a] == 0.0) return false;
  std::vector<int> out(order, order + N);
  for (int o = 0; o < 8; o += 2) {
    const int m = 7 - o;
    if (ob[o + 1] - ob[o] != ob[m + 1] - ob[m]) return false;
    for (int k = 0; k < ob[o + 1] - ob[o]; ++k) {
      const double *a = dirs + 4 * order[ob[o] + k];
      int mate = -1;
      for (int j = ob[m]; j < ob[m + 1] && mate < 0; ++j) {
        const double *b = dirs + 4 * order[j];
        if (std::fabs(a[0] + b[0]) < 1e-12 && std::fabs(a[1] + b[1]) < 1e-12 && std::fabs(a[2] + b[2]) < 1e-12)
          mate = order[j];
      }
      if (mate < 0) return false;
      out[ob[m] + k] = mate;
    }
  }
  std::copy(out.begin(), out.end(), order);
  return true;
}

// Whether the node-ray parts of two templates (of antipodal directions) are
// exact mirror images, in the sense of mirror_templates for the cell rays.
template <typename R>
inline bool mirror_node_templates(const unsigned char *ta, const unsigned char *tb, int B) {
  const TplLayout L = tpl_layout<R>(B);
  const TplEvent<R> *ea = reinterpret_cast<const TplEvent<R> *>(ta + L.nev);
  const TplEvent<R> *eb = reinterpret_cast<const TplEvent<R> *>(tb + L.nev);
  double scale = 0.0;
  for (int e = 0; e < 3 * B; ++e) scale = std::max(scale, std::fabs((double)ea[e].len));
  for (int e = 0; e < 3 * B; ++e) {
    const double la = ea[e].len, lb = eb[e].len;
    if (std::fabs(la) <= 1e-9 * scale && std::fabs(lb) <= 1e-9 * scale) continue;
    if (ea[e].off != -eb[e].off) return false;
    if (std::fabs(la - lb) > 1e-6 * std::fabs(la)) return false;
  }
  if (std::memcmp(ta + L.npos, tb + L.npos, 3 * (B + 1) * 2) != 0) return false;
  return exit_rows_match<R>(reinterpret_cast<const int16_t *>(ta + L.npos), ta + L.nk, ta + L.nw, tb + L.nk,
                            tb + L.nw, B + 1);
}

// Whether the cell-ray parts of two templates (of antipodal directions) are
// exact mirror images: equal event lengths (relative 1e-6) with negated
// offsets, zero-length tie segments aside, identical exit-event tables, and
// equal exit tables on the rows a ray can exit through.  Near-ties of plane crossings (|n_a| equal to the last bit, as on
// the unrotated HEALPix rings at 45 degrees) can be ordered differently for
// a direction and its antipode; such pairs fail the test.
template <typename R>
inline bool mirror_templates(const unsigned char *ta, const unsigned char *tb, int B) {
  const TplLayout L = tpl_layout<R>(B);
  const TplEvent<R> *ea = reinterpret_cast<const TplEvent<R> *>(ta + L.cev);
  const TplEvent<R> *eb = reinterpret_cast<const TplEvent<R> *>(tb + L.cev);
  double scale = 0.0;
  for (int e = 0; e < 3 * B; ++e) scale = std::max(scale, std::fabs((double)ea[e].len));
  for (int e = 0; e < 3 * B; ++e) {
    const double la = ea[e].len, lb = eb[e].len;
    // zero-length segments between tied interior crossings may sit in
    // either neighbouring cell: they change nothing
    if (std::fabs(la) <= 1e-9 * scale && std::fabs(lb) <= 1e-9 * scale) continue;
    if (ea[e].off != -eb[e].off) return false;
    if (std::fabs(la - lb) > 1e-6 * std::fabs(la)) return false;
  }
  if (std::memcmp(ta + L.cpos, tb + L.cpos, 3 * B * 2) != 0) return false;
  return exit_rows_match<R>(reinterpret_cast<const int16_t *>(ta + L.cpos), ta + L.ck, ta + L.cw, tb + L.ck,
                            tb + L.cw, B);
}

// Whether the paired cell pass may march an antipodal pair as one mirrored
// pair: the cell c in d and the mirror cell B - 1 - c in -d then share their
// upwind-frame coordinates, exit and face index, which needs every sign to
// flip (a zero component counts as positive, so a direction with one keeps
// that sign in its antipode) and the cell-ray templates to be exact mirrors.
template <typename R>
inline bool mirrored_cell_pair(const unsigned char *ta, const unsigned char *tb, int B) {
  const TplHead<R> *ha = reinterpret_cast<const TplHead<R> *>(ta);
  const TplHead<R> *hb = reinterpret_cast<const TplHead<R> *>(tb);
  for (int a = 0; a < 3; ++a)
    if (ha->sgn[a] != -hb->sgn[a]) return false;
  return mirror_templates<R>(ta, tb, B);
}

// Node order of the paired face pass for one template.  A node ray starts
// on a block's downwind face normal to axis a, at node (ub, uc), code
// a (B+1)^2 + ub (B+1) + uc.  The face pass hands consecutive entries of an
// order to the lanes of a warp, which march in lockstep for as many steps
// as their longest ray: in row order their rays differ in length by up to a
// block edge's worth of events (0.59 of the lane-steps useful on the
// 192-direction set).  out[a (B+1)^2 + k], a = 0..2: the face's nodes as
// ub (B+1) + uc by the index of their ray's exit event (ties by node
// index), each within 31 places of its rank in that order; then
// out[3 (B+1)^2 + k]: the codes of all three faces merged the same way,
// for items whose three downwind faces are all computed.
template <typename R>
inline void node_order(const unsigned char *tpl, int B, uint16_t *out) {
  const TplLayout L = tpl_layout<R>(B);
  const int16_t *npos = reinterpret_cast<const int16_t *>(tpl + L.npos);
  const TplHead<R> *hd = reinterpret_cast<const TplHead<R> *>(tpl);
  const int N1 = B + 1, NN = N1 * N1;
  // exit event index and tile bank group of every node code: a ray's
  // 16-byte tile entries sit in group (c0 + c1 + c2) mod 8 of the eight
  // (the tile's strides are 1 mod 8), c its start cell, and eight lanes of
  // a warp load in one wavefront only where their groups differ
  std::vector<int> last(3 * NN), grp(3 * NN);
  for (int a = 0; a < 3; ++a)
    for (int r = 0; r < NN; ++r) {
      const int ub = r / N1, uc = r % N1;
      // upwind-frame node coordinates: B along the face's axis
      const int Lq[3] = {a == 0 ? B : ub, a == 1 ? B : (a == 0 ? ub : uc), a == 2 ? B : uc};
      last[a * NN + r] = std::min({(int)npos[Lq[0]], (int)npos[N1 + Lq[1]], (int)npos[2 * N1 + Lq[2]]});
      int c = 0;
      for (int b = 0; b < 3; ++b) c += hd->sgn[b] > 0 ? Lq[b] - 1 : B - Lq[b];
      grp[a * NN + r] = ((c % 8) + 8) % 8;
    }
  // codes [c0, c0 + n) sorted by exit event, then each position takes the
  // earliest of the next 32 whose group differs from the 7 placed before it
  // (else the earliest), which keeps the length order to within a few places
  auto order = [&](int c0, int n, uint16_t *o, int sub) {
    std::vector<int> sorted(n);
    for (int k = 0; k < n; ++k) sorted[k] = c0 + k;
    std::stable_sort(sorted.begin(), sorted.end(), [&](int x, int y) { return last[x] < last[y]; });
    std::vector<char> used(n, 0);
    std::vector<int> placed(n);
    int head = 0;
    for (int p = 0; p < n; ++p) {
      while (head < n && used[head]) ++head;
      int pick = head;
      for (int c = head; c < n && c < head + 32; ++c) {
        if (used[c]) continue;
        bool distinct = true;
        for (int k = 1; k <= 7 && k <= p; ++k)
          if (grp[placed[p - k]] == grp[sorted[c]]) distinct = false;
        if (distinct) {
          pick = c;
          break;
        }
      }
      used[pick] = 1;
      placed[p] = sorted[pick];
      o[p] = (uint16_t)(placed[p] - sub);
    }
  };
  for (int a = 0; a < 3; ++a) order(a * NN, NN, out + a * NN, a * NN);
  order(0, 3 * NN, out + 3 * NN, 0);
}

// Face-pass schedule: level L of block b in octant o is b's upwind-ordered
// index sum; one item = (block, up to `group` directions of one octant), or
// up to level_group[L] directions on level L when that table is given.
// paired: only the octants with a non-negative x component are listed; an
// item then also stands for the point-mirrored block (nb - 1 - b per axis,
// at the same level) with the antipodal directions from mirror_begin on
// (the order of mirror_octant_order).
// Writes level_off[0..nlevels] and, when items != nullptr, the items.
// Returns the number of items, or -1 if it exceeds `cap`.
inline long long build_schedule(const int nb[3], const int ob[9], int group, FaceItem *items, long long cap,
                                int *level_off, const int *level_group = nullptr, bool paired = false) {
  const int nlevels = nb[0] + nb[1] + nb[2] - 2;
  // visit(L, f) calls f(block, d0, count, mirror d0, octant) for every item of level L
  auto visit = [&](int L, auto &&f) {
    for (int o = 0; o < 8; o += paired ? 2 : 1) {
      if (ob[o + 1] == ob[o]) continue;
      const int mshift = ob[7 - o] - ob[o];  // paired: antipode of d is d + mshift
      const int s[3] = {(o & 1) ? -1 : 1, (o & 2) ? -1 : 1, (o & 4) ? -1 : 1};
      for (int bz = 0; bz < nb[2]; ++bz)
        for (int by = 0; by < nb[1]; ++by)
          for (int bx = 0; bx < nb[0]; ++bx) {
            const int bb[3] = {bx, by, bz};
            int lv = 0, live = 0;
            for (int a = 0; a < 3; ++a) {
              lv += s[a] > 0 ? bb[a] : nb[a] - 1 - bb[a];
              live += (s[a] > 0 ? bb[a] + 1 < nb[a] : bb[a] > 0) ? 1 : 0;  // downwind neighbour exists
            }
            // a block whose downwind faces all lie on the domain boundary
            // produces nothing any block reads
            if (lv != L || live == 0) continue;
            const int id = (bz * nb[1] + by) * nb[0] + bx;
            const int g = level_group ? level_group[L] : group;
            for (int d0 = ob[o]; d0 < ob[o + 1]; d0 += g) f(id, d0, std::min(g, ob[o + 1] - d0), d0 + mshift, o);
          }
    }
  };
  long long total = 0;
  for (int L = 0; L < nlevels; ++L) {
    level_off[L] = (int)total;
    visit(L, [&](int, int, int, int, int) { ++total; });
  }
  level_off[nlevels] = (int)total;
  if (total > cap) return -1;
  if (!items) return total;
  long long k = 0;
  for (int L = 0; L < nlevels; ++L)
    visit(L, [&](int id, int d0, int cnt, int m0, int o) { items[k++] = {id, d0, cnt, paired ? m0 : 0, o}; });
  return k;
}

}  // namespace geom
}  // namespace vet
