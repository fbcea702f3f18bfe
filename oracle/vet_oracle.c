/*
 * vet_oracle.c -- plain, slow, FP64 CPU oracle for the non-local Variable
 * Eddington Tensor (VET) closure of VETTAM (Menon et al. 2022, MNRAS;
 * arXiv 2202.08778).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes, in the paper's order (Sec. 2.2.5, "Computing the
 * Eddington Tensor"):
 *   1. a HEALPix set of N = 12 nside^2 equal-area directions n_k with equal
 *      weights w_k = 4 pi / N, optionally rotated (Sec. 2.2.5, App. B);
 *   2. the formal solution of the time-independent gray transfer equation
 *      dI/ds = kappa (S - I)  (Eq. 14, "RTeq"; kappa here already includes
 *      the density factor rho) along every direction, by hybrid
 *      characteristics on a grid split into cubic blocks (reading below);
 *   3. the angular quadratures E, F_i, P_ij (Eqs. 10-12 and the discrete
 *      sums of Sec. 2.2.5, Eqs. 55-56, with c = 1);
 *   4. the Eddington tensor f_ij = P_ij / E (Eq. 13, "closure").
 *
 * Reading of "hybrid characteristics" (the paper names the method and cites
 * Buntemeyer et al. 2016 but gives no algorithm):
 *   - inside a block, long characteristics: the intensity at a point p is the
 *     exact solution of Eq. 14 along the straight backward ray p - t n,
 *     integrated over piecewise-constant kappa, S cells, starting from the
 *     point q where the ray leaves the block through one of its upwind faces;
 *   - between blocks, short characteristics: the intensity at q is bilinearly
 *     interpolated from intensities the upwind neighbour block computed at
 *     the lattice points (cell corners) of the face it shares, (B+1)^2 nodes
 *     per face, each of them obtained the same way (a long characteristic from
 *     the node back to that neighbour's own upwind faces);
 *   - on a domain face the entering intensity is the boundary value
 *     Ib[face][k] (constant over the face for each direction);
 *   - a ray that reaches several upwind faces at the same parameter leaves
 *     through the lowest axis (x, then y, then z);
 *   - a direction component equal to +0 or -0 counts as positive;
 *   - a point that lies on a cell face is in the cell it enters when moving
 *     backward along the ray.
 *
 * Geometry is in cell units: cell (i,j,k) spans [i,i+1]x[j,j+1]x[k,k+1] and
 * its centre is (i+1/2, j+1/2, k+1/2); physical lengths are cell units times
 * h.  Arrays are [z][y][x] row-major (x fastest).  Boundary faces are indexed
 * 0:x-low 1:x-high 2:y-low 3:y-high 4:z-low 5:z-high.
 *
 * Parity: pinned by the tests against closed forms (uniform media, beams in
 * vacuum, pure absorbers, emitting slabs), the HEALPix ring closed forms and
 * quadrature identities, and a brute-force fine-step ray integrator written
 * separately in Python.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 2

typedef struct {
  int nx, ny, nz; /* cells along x, y, z */
  int B;          /* cubic block edge in cells; must divide nx, ny, nz */
  double h;       /* cell edge length */
} ora_grid;

/* ------------------------------------------------------------------------ */
/* 1. Directions: HEALPix ring-scheme pixel centres (Gorski et al. 2005),    */
/*    rotated by the unit quaternion q = (w, x, y, z).                       */
/* ------------------------------------------------------------------------ */

static void quat_to_matrix(const double q_in[4], double R[3][3]) {
  double w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];
  double s = sqrt(w * w + x * x + y * y + z * z);
  w /= s; x /= s; y /= s; z /= s;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* dirs: [N][4] = (nx, ny, nz, w).  Pixel order: ring by ring from the north
 * pole, increasing phi within a ring.  q == NULL means no rotation. */
int ora_healpix(int nside, const double *q, double *dirs) {
  if (nside < 1 || (nside & (nside - 1)) != 0 || !dirs) return ORA_EINVAL;
  const double PI = 3.14159265358979323846;
  const int N = 12 * nside * nside;
  const double w = 4.0 * PI / N;
  double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (q) quat_to_matrix(q, R);
  int p = 0;
  for (int i = 1; i <= 4 * nside - 1; ++i) {
    double z, phi0, dphi;
    int npix;
    if (i < nside) { /* north polar cap */
      z = 1.0 - (double)i * i / (3.0 * nside * nside);
      npix = 4 * i; dphi = PI / (2.0 * i); phi0 = 0.5 * dphi;
    } else if (i <= 3 * nside) { /* equatorial belt */
      z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside);
      int s = (i - nside + 1) % 2;
      npix = 4 * nside; dphi = PI / (2.0 * nside);
      /* phi_j = dphi (j - s/2), j = 1..4 nside: first pixel at dphi (1 - s/2) */
      phi0 = dphi * (1.0 - 0.5 * s);
    } else { /* south polar cap: mirror of ring 4 nside - i */
      int ii = 4 * nside - i;
      z = -(1.0 - (double)ii * ii / (3.0 * nside * nside));
      npix = 4 * ii; dphi = PI / (2.0 * ii); phi0 = 0.5 * dphi;
    }
    double st = sqrt((1.0 - z) * (1.0 + z));
    for (int j = 0; j < npix; ++j) {
      double phi = phi0 + j * dphi;
      double v[3] = {st * cos(phi), st * sin(phi), z};
      for (int a = 0; a < 3; ++a)
        dirs[4 * p + a] = R[a][0] * v[0] + R[a][1] * v[1] + R[a][2] * v[2];
      dirs[4 * p + 3] = w;
      ++p;
    }
  }
  return p == N ? ORA_OK : ORA_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* 2. Formal solution of Eq. 14 by hybrid characteristics.                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  const ora_grid *g;
  const double *kappa, *S;
  int nbx, nby, nbz;
  int nnode;        /* (B+1)^2 */
  double n[3];      /* direction */
  double an[3];     /* |n_a| */
  int sgn[3];       /* +1 if n_a >= 0 else -1 */
  double *faces;    /* [block][axis][(B+1)^2] outgoing face nodes, this dir */
  double Ib[6];     /* boundary intensities of this direction */
} sweep_t;

typedef struct { long cell; double len; } seg_t;

/* Cell index along one axis entered when moving backward from coordinate x. */
static int entered_cell(double x, int sgn) {
  if (sgn > 0) return (int)ceil(x) - 1;
  return (int)floor(x);
}

/* Trace the backward ray from point p (cell units) through block (bx,by,bz):
 * fills seg[] with the cells crossed, nearest first, and returns the count;
 * *t_exit and *axis_exit describe where the ray leaves the block. */
static int block_ray(const sweep_t *sw, const double p[3], const int blk[3], seg_t *seg,
                     double *t_exit, int *axis_exit) {
  const ora_grid *g = sw->g;
  const int B = g->B;
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = (double)blk[a] * B;
    hi[a] = lo[a] + B;
  }
  /* parameter at which each upwind face plane is reached */
  double te = INFINITY;
  int ae = 0;
  for (int a = 0; a < 3; ++a) {
    double d = sw->sgn[a] > 0 ? p[a] - lo[a] : hi[a] - p[a];
    double t;
    if (d <= 0.0) t = 0.0;
    else if (sw->an[a] == 0.0) t = INFINITY;
    else t = d / sw->an[a];
    if (t < te) { te = t; ae = a; } /* strict: lowest axis wins ties */
  }
  *t_exit = te;
  *axis_exit = ae;
  if (te == 0.0) return 0;
  /* DDA (Amanatides & Woo 1987) from p backward to te */
  /* tnext[a]: parameter of the next cell-face plane of axis a, recomputed
   * from the exact integer plane so that the plane of the exit face gives
   * exactly t_exit */
  int c[3];
  double tnext[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = entered_cell(p[a], sw->sgn[a]);
    double plane = sw->sgn[a] > 0 ? (double)c[a] : (double)(c[a] + 1);
    tnext[a] = sw->an[a] == 0.0 ? INFINITY : fabs(p[a] - plane) / sw->an[a];
  }
  int ns = 0;
  double tprev = 0.0;
  for (;;) {
    int a = 0;
    if (tnext[1] < tnext[a]) a = 1;
    if (tnext[2] < tnext[a]) a = 2;
    long cell = ((long)c[2] * g->ny + c[1]) * g->nx + c[0];
    if (tnext[a] >= te) {
      seg[ns].cell = cell; seg[ns].len = te - tprev; ++ns;
      break;
    }
    seg[ns].cell = cell; seg[ns].len = tnext[a] - tprev; ++ns;
    tprev = tnext[a];
    c[a] -= sw->sgn[a];
    double plane = sw->sgn[a] > 0 ? (double)c[a] : (double)(c[a] + 1);
    tnext[a] = fabs(p[a] - plane) / sw->an[a];
  }
  return ns;
}

static double face_node(const sweep_t *sw, long blk_id, int axis, int u, int v) {
  const int B = sw->g->B;
  return sw->faces[((size_t)blk_id * 3 + axis) * sw->nnode + (size_t)u * (B + 1) + v];
}

/* Intensity entering at q on the upwind face (axis ae) of block blk. */
static double entry_intensity(const sweep_t *sw, const double q[3], const int blk[3], int ae) {
  const int B = sw->g->B;
  int nb[3] = {blk[0], blk[1], blk[2]};
  nb[ae] -= sw->sgn[ae];
  int nblk[3] = {sw->nbx, sw->nby, sw->nbz};
  if (nb[ae] < 0 || nb[ae] >= nblk[ae]) {
    int face = 2 * ae + (sw->sgn[ae] > 0 ? 0 : 1);
    return sw->Ib[face];
  }
  /* the two in-plane axes, lower index first */
  int b = ae == 0 ? 1 : 0;
  int c = ae == 2 ? 1 : 2;
  double ub = q[b] - (double)blk[b] * B;
  double uc = q[c] - (double)blk[c] * B;
  ub = ub < 0 ? 0 : (ub > B ? B : ub);
  uc = uc < 0 ? 0 : (uc > B ? B : uc);
  int i0 = (int)floor(ub); if (i0 > B - 1) i0 = B - 1;
  int j0 = (int)floor(uc); if (j0 > B - 1) j0 = B - 1;
  double fb = ub - i0, fc = uc - j0;
  long nid = ((long)nb[2] * sw->nby + nb[1]) * sw->nbx + nb[0];
  return (1 - fb) * (1 - fc) * face_node(sw, nid, ae, i0, j0) +
         fb * (1 - fc) * face_node(sw, nid, ae, i0 + 1, j0) +
         (1 - fb) * fc * face_node(sw, nid, ae, i0, j0 + 1) +
         fb * fc * face_node(sw, nid, ae, i0 + 1, j0 + 1);
}

/* Intensity at point p inside (or on the boundary of) block blk. */
static double point_intensity(const sweep_t *sw, const double p[3], const int blk[3], seg_t *seg) {
  double te;
  int ae;
  int ns = block_ray(sw, p, blk, seg, &te, &ae);
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = p[a] - te * sw->n[a];
  double I = entry_intensity(sw, q, blk, ae);
  const double h = sw->g->h;
  /* integrate Eq. 14 forward from q to p: exact update per constant cell */
  for (int s = ns - 1; s >= 0; --s) {
    double k = sw->kappa[seg[s].cell], Sc = sw->S[seg[s].cell];
    I = Sc + (I - Sc) * exp(-k * seg[s].len * h);
  }
  return I;
}

/* One direction: sweep the blocks in an upwind-first order, filling the face
 * nodes of each block and the cell intensities I[cells]. */
static void sweep_direction(sweep_t *sw, double *I, seg_t *seg) {
  const ora_grid *g = sw->g;
  const int B = g->B;
  int nblk[3] = {sw->nbx, sw->nby, sw->nbz};
  int order[3][2]; /* start, step per axis */
  for (int a = 0; a < 3; ++a) {
    order[a][0] = sw->sgn[a] > 0 ? 0 : nblk[a] - 1;
    order[a][1] = sw->sgn[a] > 0 ? 1 : -1;
  }
  for (int kz = 0; kz < nblk[2]; ++kz)
    for (int ky = 0; ky < nblk[1]; ++ky)
      for (int kx = 0; kx < nblk[0]; ++kx) {
        int blk[3] = {order[0][0] + kx * order[0][1], order[1][0] + ky * order[1][1],
                      order[2][0] + kz * order[2][1]};
        long bid = ((long)blk[2] * sw->nby + blk[1]) * sw->nbx + blk[0];
        /* downwind face nodes, one face per axis */
        for (int a = 0; a < 3; ++a) {
          int b = a == 0 ? 1 : 0;
          int c = a == 2 ? 1 : 2;
          double plane = (double)blk[a] * B + (sw->sgn[a] > 0 ? B : 0);
          for (int u = 0; u <= B; ++u)
            for (int v = 0; v <= B; ++v) {
              double p[3];
              p[a] = plane;
              p[b] = (double)blk[b] * B + u;
              p[c] = (double)blk[c] * B + v;
              sw->faces[((size_t)bid * 3 + a) * sw->nnode + (size_t)u * (B + 1) + v] =
                  point_intensity(sw, p, blk, seg);
            }
        }
        /* cell centres */
        if (I) {
          for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
              for (int i = 0; i < B; ++i) {
                int ci = blk[0] * B + i, cj = blk[1] * B + j, ck = blk[2] * B + k;
                double p[3] = {ci + 0.5, cj + 0.5, ck + 0.5};
                I[((long)ck * g->ny + cj) * g->nx + ci] = point_intensity(sw, p, blk, seg);
              }
        }
      }
}

typedef struct {
  const ora_grid *g;
  const double *dirs, *kappa, *S, *Ib;
  double *I_out;
  int ndir, tid, nthreads, status;
} job_t;

static void *trace_worker(void *arg) {
  job_t *jb = (job_t *)arg;
  const ora_grid *g = jb->g;
  const int B = g->B;
  sweep_t sw;
  memset(&sw, 0, sizeof sw);
  sw.g = g; sw.kappa = jb->kappa; sw.S = jb->S;
  sw.nbx = g->nx / B; sw.nby = g->ny / B; sw.nbz = g->nz / B;
  sw.nnode = (B + 1) * (B + 1);
  size_t nblocks = (size_t)sw.nbx * sw.nby * sw.nbz;
  sw.faces = (double *)malloc(nblocks * 3 * sw.nnode * sizeof(double));
  seg_t *seg = (seg_t *)malloc((size_t)(3 * B + 4) * sizeof(seg_t));
  if (!sw.faces || !seg) { jb->status = ORA_ENOMEM; free(sw.faces); free(seg); return NULL; }
  const long ncell = (long)g->nx * g->ny * g->nz;
  for (int k = jb->tid; k < jb->ndir; k += jb->nthreads) {
    for (int a = 0; a < 3; ++a) {
      sw.n[a] = jb->dirs[4 * k + a];
      sw.an[a] = fabs(sw.n[a]);
      sw.sgn[a] = signbit(sw.n[a]) && sw.n[a] != 0.0 ? -1 : 1;
    }
    for (int f = 0; f < 6; ++f) sw.Ib[f] = jb->Ib ? jb->Ib[(size_t)f * jb->ndir + k] : 0.0;
    sweep_direction(&sw, jb->I_out + (size_t)k * ncell, seg);
  }
  free(sw.faces);
  free(seg);
  return NULL;
}

/* Hybrid-characteristics formal solution for ndir directions.
 *   dirs  [ndir][4] (nx, ny, nz, w), kappa and S [cells] (kappa per unit
 *   length, already times rho), Ib [6][ndir] or NULL (vacuum),
 *   I_out [ndir][cells].  nthreads >= 1 splits the directions. */
int ora_trace(const ora_grid *g, const double *dirs, int ndir, const double *kappa, const double *S,
              const double *Ib, double *I_out, int nthreads) {
  if (!g || !dirs || !kappa || !S || !I_out || ndir < 1) return ORA_EINVAL;
  if (g->B < 1 || g->nx < 1 || g->ny < 1 || g->nz < 1) return ORA_EINVAL;
  if (g->nx % g->B || g->ny % g->B || g->nz % g->B || !(g->h > 0)) return ORA_EINVAL;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > ndir) nthreads = ndir;
  job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return ORA_ENOMEM; }
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job_t){g, dirs, kappa, S, Ib, I_out, ndir, t, nthreads, ORA_OK};
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, trace_worker, &jobs[t]);
  trace_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  int st = ORA_OK;
  for (int t = 0; t < nthreads; ++t)
    if (jobs[t].status != ORA_OK) st = jobs[t].status;
  free(jobs);
  free(th);
  return st;
}

/* ------------------------------------------------------------------------ */
/* 3. Angular quadratures (Sec. 2.2.5 sums; Eqs. 10-12 with c = 1):            */
/*    E = sum_k w_k I_k, F_i = sum_k w_k I_k n_ik,                            */
/*    P_ij = sum_k w_k I_k n_ik n_jk.                                         */
/*    M [10][cells] = E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz.            */
/* ------------------------------------------------------------------------ */
int ora_moments(const double *I, const double *dirs, int ndir, long ncell, double *M) {
  if (!I || !dirs || !M || ndir < 1 || ncell < 0) return ORA_EINVAL;
  for (long c = 0; c < ncell; ++c) {
    double acc[10] = {0};
    for (int k = 0; k < ndir; ++k) {
      const double *d = dirs + 4 * k;
      double wI = d[3] * I[(size_t)k * ncell + c];
      acc[0] += wI;
      acc[1] += wI * d[0];
      acc[2] += wI * d[1];
      acc[3] += wI * d[2];
      acc[4] += wI * d[0] * d[0];
      acc[5] += wI * d[1] * d[1];
      acc[6] += wI * d[2] * d[2];
      acc[7] += wI * d[0] * d[1];
      acc[8] += wI * d[0] * d[2];
      acc[9] += wI * d[1] * d[2];
    }
    for (int m = 0; m < 10; ++m) M[(size_t)m * ncell + c] = acc[m];
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* 4. Closure (Eq. 13): f_ij = P_ij / E.  Cells whose E does not exceed       */
/*    E_floor = floor_rel * max_cells E receive the isotropic tensor I/3 and */
/*    flag[c] = 1 (E = 0 happens where no radiation reaches a cell).         */
/*    f [6][cells] = xx, yy, zz, xy, xz, yz.                                  */
/* ------------------------------------------------------------------------ */
int ora_closure(const double *M, long ncell, double floor_rel, double *f, unsigned char *flag) {
  if (!M || !f || ncell < 0) return ORA_EINVAL;
  double emax = 0.0;
  for (long c = 0; c < ncell; ++c)
    if (M[c] > emax) emax = M[c];
  double efloor = floor_rel * emax;
  for (long c = 0; c < ncell; ++c) {
    double E = M[c];
    int iso = !(E > efloor);
    for (int m = 0; m < 6; ++m) {
      double v = iso ? (m < 3 ? 1.0 / 3.0 : 0.0) : M[(size_t)(4 + m) * ncell + c] / E;
      f[(size_t)m * ncell + c] = v;
    }
    if (flag) flag[c] = (unsigned char)iso;
  }
  return ORA_OK;
}

/* Number of segments each backward ray crosses, for every cell and
 * direction (the work measure of the method): returns the sum over cells and
 * directions of cell-ray segments and, in *face_segs, of face-node-ray
 * segments.  Geometry only; kappa and S are not read. */
long long ora_count_segments(const ora_grid *g, const double *dirs, int ndir, long long *face_segs) {
  if (!g || !dirs || ndir < 1 || g->B < 1 || g->nx % g->B || g->ny % g->B || g->nz % g->B) return -1;
  const int B = g->B;
  sweep_t sw;
  memset(&sw, 0, sizeof sw);
  sw.g = g;
  sw.nbx = g->nx / B; sw.nby = g->ny / B; sw.nbz = g->nz / B;
  seg_t *seg = (seg_t *)malloc((size_t)(3 * B + 4) * sizeof(seg_t));
  if (!seg) return -1;
  long long cells = 0, faces = 0;
  int blk[3] = {0, 0, 0};
  for (int k = 0; k < ndir; ++k) {
    for (int a = 0; a < 3; ++a) {
      sw.n[a] = dirs[4 * k + a];
      sw.an[a] = fabs(sw.n[a]);
      sw.sgn[a] = signbit(sw.n[a]) && sw.n[a] != 0.0 ? -1 : 1;
    }
    double te;
    int ae;
    for (int kk = 0; kk < B; ++kk)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          double p[3] = {i + 0.5, j + 0.5, kk + 0.5};
          cells += block_ray(&sw, p, blk, seg, &te, &ae);
        }
    for (int a = 0; a < 3; ++a) {
      int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
      for (int u = 0; u <= B; ++u)
        for (int v = 0; v <= B; ++v) {
          double p[3];
          p[a] = sw.sgn[a] > 0 ? B : 0;
          p[b] = u;
          p[c] = v;
          faces += block_ray(&sw, p, blk, seg, &te, &ae);
        }
    }
  }
  free(seg);
  long long nb = (long long)sw.nbx * sw.nby * sw.nbz;
  if (face_segs) *face_segs = faces * nb;
  return cells * nb;
}
