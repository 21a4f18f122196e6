/*
 * fd_oracle.c -- plain FP64 CPU oracle for the explicit finite-difference sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Called through ctypes by oracle/core.py from the
 * tests, from __graft_entry__.smoke() and from the CPU-baseline leg of bench.py.
 * It shares no code with the CUDA library.  Everything is evaluated in double,
 * one grid point at a time, in the order the scheme is written; there is no
 * blocking, fusion or reordering.  OpenMP only splits the outer loops of a
 * point-wise update (each point is still computed by the same expression).
 *
 * Arrays are dense, C order, interior only (no halo):
 *   ndim = 3: [n0][n1][n2]     ndim = 2: [n0][n1]      (last axis contiguous)
 * Axis d has n[d] nodes at coordinates i*h[d], i = 0..n[d]-1.
 * Values outside the grid are taken as zero (zero halo), or, in the diffusion
 * sweep's odd-reflection mode (bc = 1), as the negated value mirrored about
 * the nearest boundary node: u(-k) = -u(k) and u(n-1+k) = -u(n-1-k) along the
 * axis that leaves the grid (the stencil is a star: one axis at a time).
 *
 * Method (thesis §5.1.2 for the diffusion problem; §6.2.1 names the acoustic
 * operator with sources and receivers as the seismic operator the OPS backend
 * could not run, so its discrete form is the standard second-order leapfrog):
 *
 *   L u (i)  = Σ_d  (1/h_d²) Σ_{k=-r..r} w_|k| u(i + k e_d)        (r = so/2)
 *
 *   diffusion (forward Euler; §2.1.1's `subdomain=grid.interior`: interior nodes
 *   only, boundary nodes fixed; or, without that subdomain (interior = 0), every
 *   node, the values outside the grid zero):
 *     u^{n+1} = u^n + ν dt L u^n
 *
 *   acoustic (all nodes, σ = damp·dt/2):
 *     m (u^{n+1} - 2u^n + u^{n-1}) + σ (u^{n+1} - u^{n-1}) = dt² L u^n
 *     then   u^{n+1}(node) += wgt · dt² · s_j(t_n) / m(node)   (2^D corners of source j)
 *     and    rec_k(t_{n+1}) = Σ_corners wgt · u^{n+1}(node)
 *
 * Multilinear corner weights of a point c (physical coordinates): per axis
 * x = c_d/h_d, i = floor(x), f = x - i; a point on the last node uses
 * i = n-2, f = 1; x within 1e-9·(n-1) outside [0, n-1] is snapped onto the
 * end node, x further outside is an error.  Corner bits b_d select
 * node i+b_d with factor f (b_d = 1) or 1-f (b_d = 0); axis 0 is the most
 * significant bit of the corner number.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

typedef struct {
  int ndim;
  int64_t n[3];   /* nodes per axis (axes >= ndim unused) */
  int64_t st[3];  /* element stride per axis */
  int64_t e[3];   /* loop extents in 3-D form: 2-D grids get e = {1, n0, n1} */
  int64_t total;
} grid_t;

static int grid_init(grid_t *g, int ndim, const int64_t *shape) {
  if (ndim != 2 && ndim != 3) return OR_EINVAL;
  g->ndim = ndim;
  g->total = 1;
  for (int d = 0; d < ndim; ++d) {
    if (shape[d] < 1) return OR_EINVAL;
    g->n[d] = shape[d];
    g->total *= shape[d];
  }
  int64_t s = 1;
  for (int d = ndim - 1; d >= 0; --d) {
    g->st[d] = s;
    s *= g->n[d];
  }
  if (ndim == 3) {
    for (int d = 0; d < 3; ++d) g->e[d] = g->n[d];
  } else {
    g->e[0] = 1; g->e[1] = g->n[0]; g->e[2] = g->n[1];
  }
  return OR_OK;
}

/* multi-index of loop position (a, b, c) */
static void point_index(const grid_t *g, int64_t a, int64_t b, int64_t c,
                        int64_t *idx) {
  if (g->ndim == 3) { idx[0] = a; idx[1] = b; idx[2] = c; }
  else { idx[0] = b; idx[1] = c; }
}

/* value of u at axis-d index j of the line through flat index p (whose axis-d
 * index is i): inside the grid the node value; outside, 0 (bc = 0) or the odd
 * mirror image about the boundary node (bc = 1) */
static double neighbour(const double *u, const grid_t *g, int d, int64_t i, int64_t j,
                        int64_t p, int bc) {
  const int64_t n = g->n[d];
  if (j >= 0 && j < n) return u[p + (j - i) * g->st[d]];
  if (bc == 0) return 0.0;
  const int64_t m = j < 0 ? -j : 2 * (n - 1) - j;   /* mirror index */
  return -u[p + (m - i) * g->st[d]];
}

/* L u at the point with multi-index idx and flat index p, straight from the
 * definition */
static double lap_point(const double *u, const grid_t *g, const double *h,
                        int r, const double *w, const int64_t *idx, int64_t p, int bc) {
  double s = 0.0;
  for (int d = 0; d < g->ndim; ++d) {
    double sd = w[0] * u[p];
    for (int k = 1; k <= r; ++k) {
      double up = neighbour(u, g, d, idx[d], idx[d] + k, p, bc);
      double dn = neighbour(u, g, d, idx[d], idx[d] - k, p, bc);
      sd += w[k] * (up + dn);
    }
    s += sd / (h[d] * h[d]);
  }
  return s;
}

/* the odd mirror needs a node at distance k inside: n - 1 >= r on every axis */
static int mirror_ok(const grid_t *g, int r) {
  for (int d = 0; d < g->ndim; ++d)
    if (g->n[d] - 1 < r) return 0;
  return 1;
}

static int on_boundary(const grid_t *g, const int64_t *idx) {
  for (int d = 0; d < g->ndim; ++d)
    if (idx[d] == 0 || idx[d] == g->n[d] - 1) return 1;
  return 0;
}

int oracle_laplacian(int ndim, const int64_t *shape, const double *h, int so,
                     const double *w, const double *u, double *out) {
  grid_t g;
  if (grid_init(&g, ndim, shape) || so < 2 || so % 2) return OR_EINVAL;
  const int r = so / 2;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t a = 0; a < g.e[0]; ++a)
    for (int64_t b = 0; b < g.e[1]; ++b)
      for (int64_t c = 0; c < g.e[2]; ++c) {
        int64_t idx[3], p = (a * g.e[1] + b) * g.e[2] + c;
        point_index(&g, a, b, c, idx);
        out[p] = lap_point(u, &g, h, r, w, idx, p, 0);
      }
  return OR_OK;
}

/* Diffusion, forward Euler, interior update (u is overwritten by u^{nt});
 * bc = 0: zero outside the grid, bc = 1: odd reflection about the boundary nodes. */
int oracle_diffusion(int ndim, const int64_t *shape, const double *h, int so,
                     const double *w, double nu, double dt, int nt, int bc, int interior,
                     double *u) {
  grid_t g;
  if (grid_init(&g, ndim, shape) || so < 2 || so % 2 || nt < 0) return OR_EINVAL;
  const int r = so / 2;
  if (bc != 0 && (bc != 1 || !mirror_ok(&g, r) || !interior)) return OR_EINVAL;
  double *v = (double *)malloc(sizeof(double) * (size_t)g.total);
  if (!v) return OR_ENOMEM;
  double *cur = u, *nxt = v;
  for (int n = 0; n < nt; ++n) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t a = 0; a < g.e[0]; ++a)
      for (int64_t b = 0; b < g.e[1]; ++b)
        for (int64_t c = 0; c < g.e[2]; ++c) {
          int64_t idx[3], p = (a * g.e[1] + b) * g.e[2] + c;
          point_index(&g, a, b, c, idx);
          if (interior && on_boundary(&g, idx))
            nxt[p] = cur[p];
          else
            nxt[p] = cur[p] + nu * dt * lap_point(cur, &g, h, r, w, idx, p, bc);
        }
    double *t = cur; cur = nxt; nxt = t;
  }
  if (cur != u) memcpy(u, cur, sizeof(double) * (size_t)g.total);
  free(v);
  return OR_OK;
}

/* Multilinear corners of one point: out_node[2^ndim], out_w[2^ndim]. */
int oracle_corners(int ndim, const int64_t *shape, const double *h,
                   const double *c, int64_t *out_node, double *out_w) {
  grid_t g;
  if (grid_init(&g, ndim, shape)) return OR_EINVAL;
  int64_t i[3];
  double f[3];
  for (int d = 0; d < ndim; ++d) {
    if (g.n[d] < 2) return OR_EINVAL;
    double x = c[d] / h[d];
    const double last = (double)(g.n[d] - 1), tol = 1e-9 * last;
    if (!(x >= -tol && x <= last + tol)) return OR_EINVAL;
    if (x < 0.0) x = 0.0;       /* within tol of an end: snapped onto it */
    if (x > last) x = last;
    i[d] = (int64_t)floor(x);
    f[d] = x - (double)i[d];
    if (i[d] == g.n[d] - 1) { i[d] = g.n[d] - 2; f[d] = 1.0; }
  }
  for (int b = 0; b < (1 << ndim); ++b) {
    int64_t off = 0;
    double wt = 1.0;
    for (int d = 0; d < ndim; ++d) {
      int bit = (b >> (ndim - 1 - d)) & 1;
      off += (i[d] + bit) * g.st[d];
      wt *= bit ? f[d] : 1.0 - f[d];
    }
    out_node[b] = off;
    out_w[b] = wt;
  }
  return OR_OK;
}

static void interp_all(const double *u, int ncorner, int nrec,
                       const int64_t *node, const double *wt, double *row) {
  for (int k = 0; k < nrec; ++k) {
    double s = 0.0;
    for (int b = 0; b < ncorner; ++b)
      s += wt[k * ncorner + b] * u[node[k * ncorner + b]];
    row[k] = s;
  }
}

/*
 * Acoustic leapfrog with damping, sources and receivers.
 *   u_cur  in: u^{n0}      out: u^{n0+nt}
 *   u_prev in: u^{n0-1}    out: u^{n0+nt-1}
 *   damp   may be NULL (no damping)
 *   wavelet [nt_wav][nsrc]: s_j(t_n) for global step n (needs n0+nt <= nt_wav
 *           when nsrc > 0)
 *   rec    [nt+1][nrec] or NULL: rec[0] = interp(u^{n0}),
 *           rec[s+1] = interp(u^{n0+s+1})
 */
int oracle_acoustic(int ndim, const int64_t *shape, const double *h, int so,
                    const double *w, double dt, const double *m,
                    const double *damp, double *u_cur, double *u_prev,
                    int nsrc, const double *src_coords, int nt_wav,
                    const double *wavelet, int n0, int nrec,
                    const double *rec_coords, double *rec, int nt) {
  grid_t g;
  if (grid_init(&g, ndim, shape) || so < 2 || so % 2 || nt < 0 || n0 < 0 ||
      nsrc < 0 || nrec < 0)
    return OR_EINVAL;
  if (nsrc > 0 && (int64_t)n0 + nt > nt_wav) return OR_EINVAL;
  const int r = so / 2;
  const int nc = 1 << ndim;
  const size_t bytes = sizeof(double) * (size_t)g.total;
  int64_t *snode = NULL, *rnode = NULL;
  double *swt = NULL, *rwt = NULL, *scratch = NULL;
  int status = OR_ENOMEM;
  snode = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nsrc * nc + 1));
  swt = (double *)malloc(sizeof(double) * (size_t)(nsrc * nc + 1));
  rnode = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrec * nc + 1));
  rwt = (double *)malloc(sizeof(double) * (size_t)(nrec * nc + 1));
  scratch = (double *)malloc(bytes);
  if (!snode || !swt || !rnode || !rwt || !scratch) goto done;
  status = OR_EINVAL;
  for (int j = 0; j < nsrc; ++j)
    if (oracle_corners(ndim, shape, h, src_coords + j * ndim, snode + j * nc,
                       swt + j * nc))
      goto done;
  for (int k = 0; k < nrec; ++k)
    if (oracle_corners(ndim, shape, h, rec_coords + k * ndim, rnode + k * nc,
                       rwt + k * nc))
      goto done;
  status = OR_OK;

  double *cur = u_cur, *prv = u_prev, *nxt = scratch;
  if (rec) interp_all(cur, nc, nrec, rnode, rwt, rec);
  for (int s = 0; s < nt; ++s) {
    const int n = n0 + s;
    /* stencil update of every node */
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t a = 0; a < g.e[0]; ++a)
      for (int64_t b = 0; b < g.e[1]; ++b)
        for (int64_t c = 0; c < g.e[2]; ++c) {
          int64_t idx[3], p = (a * g.e[1] + b) * g.e[2] + c;
          point_index(&g, a, b, c, idx);
          double sigma = (damp ? damp[p] : 0.0) * dt / 2.0;
          double lap = lap_point(cur, &g, h, r, w, idx, p, 0);
          nxt[p] = (dt * dt * lap + 2.0 * m[p] * cur[p] -
                    (m[p] - sigma) * prv[p]) / (m[p] + sigma);
        }
    /* point-source injection at t_n, source by source, corner by corner */
    for (int j = 0; j < nsrc; ++j) {
      double sv = wavelet[(int64_t)n * nsrc + j];
      for (int b = 0; b < nc; ++b) {
        int64_t q = snode[j * nc + b];
        nxt[q] += swt[j * nc + b] * dt * dt * sv / m[q];
      }
    }
    /* rotate: u^{n-1} <- u^n, u^n <- u^{n+1}; the old u^{n-1} buffer is reused */
    double *t = prv; prv = cur; cur = nxt; nxt = t;
    if (rec) interp_all(cur, nc, nrec, rnode, rwt, rec + (int64_t)(s + 1) * nrec);
  }
  /* hand the final two levels back in the caller's buffers (the three
   * buffers have rotated, so save u^{n+1} before overwriting anything) */
  if (nt > 0) {
    double *c2 = (double *)malloc(bytes);
    if (!c2) { status = OR_ENOMEM; goto done; }
    memcpy(c2, cur, bytes);
    if (prv != u_prev) memmove(u_prev, prv, bytes);
    memcpy(u_cur, c2, bytes);
    free(c2);
  }
done:
  free(snode); free(swt); free(rnode); free(rwt); free(scratch);
  return status;
}
