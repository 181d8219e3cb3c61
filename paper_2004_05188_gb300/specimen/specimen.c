/*
 * Seeded synthetic atom-probe specimens (input generation only).
 *
 * This module produces the point clouds that both the CUDA path and the
 * oracle consume: float32 xyz (nm, AoS), uint8 ion type and float32 d_srf
 * (analytic distance to the specimen surface).  It contains none of the
 * spatial-statistics arithmetic.
 *
 * Specimen recipes follow the paper's synthetic benchmark section (Methods,
 * "Benchmarking all functionality with synthetic datasets"): needle-shaped
 * conical frusta filled with an fcc Al lattice (a = 0.404 nm) into which
 * spherical Al3Sc precipitates are dispersed at random.  The homogeneous
 * Poisson cylinder is the textbook random point process the paper compares
 * spatial statistics against (Suppl., "Importance of high quality random
 * number generators").
 *
 * Randomness is counter based: every draw is a keyed hash of
 * (seed, stream, counter, draw), so any lattice site or ion can be generated
 * independently of every other one, in any order, by any number of threads,
 * and the output is identical for every thread count.
 *
 * Type labels: 0 = Al, 1 = Sc, 2 = Si.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PSG_OK 0
#define PSG_ERR_ARG 1
#define PSG_ERR_OOM 2

enum { ST_POS = 1, ST_TYPE = 2, ST_KEEP = 3, ST_JIT = 4, ST_PCOUNT = 5, ST_PPOS = 6, ST_LABEL = 7 };

static inline uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static inline uint64_t draw64(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t k) {
  return mix64(mix64(mix64(seed ^ (stream * 0xd1b54a32d192ed03ULL)) + ctr) + k);
}

/* uniform in [0, 1) */
static inline double unif(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t k) {
  return (double)(draw64(seed, stream, ctr, k) >> 11) * 0x1.0p-53;
}

/* uniform in (0, 1) */
static inline double unif_open(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t k) {
  return ((double)(draw64(seed, stream, ctr, k) >> 11) + 0.5) * 0x1.0p-53;
}

/* standard normal by Box-Muller from draws (k, k+1) */
static inline double normal(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t k) {
  const double u1 = unif_open(seed, stream, ctr, k);
  const double u2 = unif(seed, stream, ctr, k + 1);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static inline uint8_t pick_type(double u, const double* cum, int n_types) {
  for (int t = 0; t < n_types - 1; ++t)
    if (u < cum[t]) return (uint8_t)t;
  return (uint8_t)(n_types - 1);
}

/* ------------------------------------------------------------------------- */
/* Homogeneous Poisson (binomial, fixed n) cylinder: radius R, height H.     */
/* ------------------------------------------------------------------------- */
int psg_cylinder(uint64_t seed, int64_t n, double R, double H, const double* type_prob, int n_types,
                 float* xyz, uint8_t* type, float* dsrf) {
  if (n < 0 || !(R > 0) || !(H > 0) || n_types < 1 || n_types > 256) return PSG_ERR_ARG;
  double cum[256];
  double acc = 0.0;
  for (int t = 0; t < n_types; ++t) {
    acc += type_prob[t];
    cum[t] = acc;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double rho = R * sqrt(unif(seed, ST_POS, (uint64_t)i, 0));
    const double phi = 6.283185307179586 * unif(seed, ST_POS, (uint64_t)i, 1);
    const double z = H * unif(seed, ST_POS, (uint64_t)i, 2);
    const float fx = (float)(rho * cos(phi)), fy = (float)(rho * sin(phi)), fz = (float)z;
    xyz[3 * i + 0] = fx;
    xyz[3 * i + 1] = fy;
    xyz[3 * i + 2] = fz;
    type[i] = pick_type(unif(seed, ST_TYPE, (uint64_t)i, 0), cum, n_types);
    const double r = sqrt((double)fx * fx + (double)fy * fy);
    double d = R - r;
    if ((double)fz < d) d = (double)fz;
    if (H - (double)fz < d) d = H - (double)fz;
    dsrf[i] = (float)d;
  }
  return PSG_OK;
}

/* ------------------------------------------------------------------------- */
/* Homogeneous Poisson cube [0, L)^3 (test clouds); dsrf = distance to faces. */
/* ------------------------------------------------------------------------- */
int psg_cube(uint64_t seed, int64_t n, double L, const double* type_prob, int n_types, float* xyz,
             uint8_t* type, float* dsrf) {
  if (n < 0 || !(L > 0) || n_types < 1 || n_types > 256) return PSG_ERR_ARG;
  double cum[256];
  double acc = 0.0;
  for (int t = 0; t < n_types; ++t) {
    acc += type_prob[t];
    cum[t] = acc;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d = L;
    for (int a = 0; a < 3; ++a) {
      const float f = (float)(L * unif(seed, ST_POS, (uint64_t)i, (uint64_t)a));
      xyz[3 * i + a] = f;
      if ((double)f < d) d = (double)f;
      if (L - (double)f < d) d = L - (double)f;
    }
    type[i] = pick_type(unif(seed, ST_TYPE, (uint64_t)i, 0), cum, n_types);
    dsrf[i] = (float)d;
  }
  return PSG_OK;
}

/* ------------------------------------------------------------------------- */
/* Needle: conical frustum, base (z = 0) radius Rb, top (z = H) radius Rt.    */
/* fcc lattice, sites thinned with probability keep, Gaussian jitter,         */
/* Poisson-dispersed spherical precipitates with log-normal radii.           */
/* ------------------------------------------------------------------------- */
typedef struct {
  double r_top;       /* tip radius at z = H (nm) */
  double half_angle;  /* shank half-angle (rad) */
  double height;      /* H (nm) */
  double a;           /* fcc lattice constant (nm) */
  double keep;        /* site retention probability */
  double sig_xy, sig_z;        /* reconstruction jitter (nm) */
  double prec_density;         /* precipitate centres per nm^3 */
  double prec_median, prec_sigma; /* log-normal radius: median (nm), sigma of ln r */
  double in_sc;                /* Sc fraction inside precipitates (rest Al) */
  double out_sc, out_si;       /* Sc and Si fractions in the matrix (rest Al) */
  uint64_t seed;
} psg_needle_t;

#define PREC_BLOCK 16.0 /* precipitate hash-block edge (nm); radii are capped here */

typedef struct {
  psg_needle_t p;
  double rb, tana, cosa;
  int64_t ni, nj, nk;   /* lattice cells along x, y, z */
  double x0, y0;        /* lattice origin in x, y */
  /* precipitates, CSR by block */
  int64_t nbx, nby, nbz;
  double bx0, by0, bz0;
  int64_t* blk_off;     /* nbx*nby*nbz + 1 */
  double* prec;         /* 4 doubles each: cx, cy, cz, r^2 */
  double rmax;          /* largest realised precipitate radius */
} needle_ctx;

static const double FCC[4][3] = {{0.0, 0.0, 0.0}, {0.5, 0.5, 0.0}, {0.5, 0.0, 0.5}, {0.0, 0.5, 0.5}};

static int64_t poisson_draw(double lam, double u) {
  /* inverse CDF by summation; lam is a few units */
  double p = exp(-lam), c = p;
  int64_t k = 0;
  while (u > c && k < 1000) {
    ++k;
    p *= lam / (double)k;
    c += p;
  }
  return k;
}

static int needle_init(needle_ctx* c, const psg_needle_t* p) {
  memset(c, 0, sizeof(*c));
  c->p = *p;
  if (!(p->r_top > 0) || !(p->height > 0) || !(p->a > 0) || p->half_angle < 0 || p->half_angle >= 1.5 ||
      p->keep < 0 || p->keep > 1)
    return PSG_ERR_ARG;
  c->tana = tan(p->half_angle);
  c->cosa = cos(p->half_angle);
  c->rb = p->r_top + p->height * c->tana;
  c->ni = (int64_t)ceil(2.0 * c->rb / p->a) + 1;
  c->nj = c->ni;
  c->nk = (int64_t)ceil(p->height / p->a) + 1;
  c->x0 = -p->a * (double)(c->ni / 2);
  c->y0 = c->x0;
  /* precipitate blocks cover the bounding box with one block of slack */
  const double B = PREC_BLOCK;
  c->bx0 = -c->rb - B;
  c->by0 = -c->rb - B;
  c->bz0 = -B;
  c->nbx = (int64_t)ceil((2.0 * c->rb + 2.0 * B) / B) + 1;
  c->nby = c->nbx;
  c->nbz = (int64_t)ceil((p->height + 2.0 * B) / B) + 1;
  const int64_t nb = c->nbx * c->nby * c->nbz;
  c->blk_off = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  if (!c->blk_off) return PSG_ERR_OOM;
  const double lam = p->prec_density * B * B * B;
  for (int64_t b = 0; b < nb; ++b)
    c->blk_off[b + 1] = c->blk_off[b] + (p->prec_density > 0 ? poisson_draw(lam, unif(p->seed, ST_PCOUNT, (uint64_t)b, 0)) : 0);
  const int64_t np = c->blk_off[nb];
  c->prec = (double*)malloc((size_t)(np > 0 ? np : 1) * 4 * sizeof(double));
  if (!c->prec) {
    free(c->blk_off);
    return PSG_ERR_OOM;
  }
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t bx = b % c->nbx, by = (b / c->nbx) % c->nby, bz = b / (c->nbx * c->nby);
    for (int64_t m = c->blk_off[b]; m < c->blk_off[b + 1]; ++m) {
      const uint64_t ctr = (uint64_t)m;
      double r = p->prec_median * exp(p->prec_sigma * normal(p->seed, ST_PPOS, ctr, 3));
      if (r > B) r = B;
      c->prec[4 * m + 0] = c->bx0 + B * ((double)bx + unif(p->seed, ST_PPOS, ctr, 0));
      c->prec[4 * m + 1] = c->by0 + B * ((double)by + unif(p->seed, ST_PPOS, ctr, 1));
      c->prec[4 * m + 2] = c->bz0 + B * ((double)bz + unif(p->seed, ST_PPOS, ctr, 2));
      c->prec[4 * m + 3] = r * r;
      if (r > c->rmax) c->rmax = r;
    }
  }
  return PSG_OK;
}

static void needle_free(needle_ctx* c) {
  free(c->blk_off);
  free(c->prec);
}

static int in_precipitate(const needle_ctx* c, double x, double y, double z) {
  const double B = PREC_BLOCK, r = c->rmax;
  const int64_t X0 = (int64_t)floor((x - r - c->bx0) / B), X1 = (int64_t)floor((x + r - c->bx0) / B);
  const int64_t Y0 = (int64_t)floor((y - r - c->by0) / B), Y1 = (int64_t)floor((y + r - c->by0) / B);
  const int64_t Z0 = (int64_t)floor((z - r - c->bz0) / B), Z1 = (int64_t)floor((z + r - c->bz0) / B);
  for (int64_t Z = Z0; Z <= Z1; ++Z)
    for (int64_t Y = Y0; Y <= Y1; ++Y)
      for (int64_t X = X0; X <= X1; ++X) {
        if (X < 0 || Y < 0 || Z < 0 || X >= c->nbx || Y >= c->nby || Z >= c->nbz) continue;
        const int64_t b = (Z * c->nby + Y) * c->nbx + X;
        for (int64_t m = c->blk_off[b]; m < c->blk_off[b + 1]; ++m) {
          const double ex = x - c->prec[4 * m], ey = y - c->prec[4 * m + 1], ez = z - c->prec[4 * m + 2];
          if (ex * ex + ey * ey + ez * ez < c->prec[4 * m + 3]) return 1;
        }
      }
  return 0;
}

/* site (i, j, k, b) -> position and inside test; returns 1 if the site lies in the frustum */
static inline int site_pos(const needle_ctx* c, int64_t i, int64_t j, int64_t k, int b, double* s) {
  const double a = c->p.a;
  s[0] = c->x0 + a * ((double)i + FCC[b][0]);
  s[1] = c->y0 + a * ((double)j + FCC[b][1]);
  s[2] = a * ((double)k + FCC[b][2]);
  if (s[2] < 0.0 || s[2] >= c->p.height) return 0;
  const double R = c->rb - s[2] * c->tana;
  return s[0] * s[0] + s[1] * s[1] < R * R;
}

static inline uint64_t site_id(const needle_ctx* c, int64_t i, int64_t j, int64_t k, int b) {
  return (uint64_t)((((k * c->nj) + j) * c->ni + i) * 4 + b);
}

static int64_t layer_count(const needle_ctx* c, int64_t k) {
  int64_t cnt = 0;
  double s[3];
  for (int64_t j = 0; j < c->nj; ++j)
    for (int64_t i = 0; i < c->ni; ++i)
      for (int b = 0; b < 4; ++b) {
        if (!site_pos(c, i, j, k, b, s)) continue;
        if (unif(c->p.seed, ST_KEEP, site_id(c, i, j, k, b), 0) < c->p.keep) ++cnt;
      }
  return cnt;
}

static void layer_fill(const needle_ctx* c, int64_t k, float* xyz, uint8_t* type, float* dsrf) {
  int64_t o = 0;
  double s[3];
  const psg_needle_t* p = &c->p;
  for (int64_t j = 0; j < c->nj; ++j)
    for (int64_t i = 0; i < c->ni; ++i)
      for (int b = 0; b < 4; ++b) {
        if (!site_pos(c, i, j, k, b, s)) continue;
        const uint64_t id = site_id(c, i, j, k, b);
        if (!(unif(p->seed, ST_KEEP, id, 0) < p->keep)) continue;
        const double x = s[0] + p->sig_xy * normal(p->seed, ST_JIT, id, 0);
        const double y = s[1] + p->sig_xy * normal(p->seed, ST_JIT, id, 2);
        const double z = s[2] + p->sig_z * normal(p->seed, ST_JIT, id, 4);
        const float fx = (float)x, fy = (float)y, fz = (float)z;
        xyz[3 * o + 0] = fx;
        xyz[3 * o + 1] = fy;
        xyz[3 * o + 2] = fz;
        const double u = unif(p->seed, ST_LABEL, id, 0);
        uint8_t t;
        if (in_precipitate(c, s[0], s[1], s[2]))
          t = (u < p->in_sc) ? 1 : 0;
        else
          t = (u < p->out_sc) ? 1 : (u < p->out_sc + p->out_si) ? 2 : 0;
        type[o] = t;
        /* analytic distance to the frustum: lateral face, bottom, top */
        const double zd = (double)fz;
        const double rho = sqrt((double)fx * fx + (double)fy * fy);
        double d = (c->rb - zd * c->tana - rho) * c->cosa;
        if (zd < d) d = zd;
        if (p->height - zd < d) d = p->height - zd;
        dsrf[o] = (float)d;
        ++o;
      }
}

/* number of z layers of lattice cells */
int64_t psg_needle_layers(const psg_needle_t* p) {
  needle_ctx c;
  if (needle_init(&c, p) != PSG_OK) return -1;
  const int64_t nk = c.nk;
  needle_free(&c);
  return nk;
}

/* ions per z layer (counts[nk]); total returned (or -1 on error) */
int64_t psg_needle_plan(const psg_needle_t* p, int64_t* counts) {
  needle_ctx c;
  if (needle_init(&c, p) != PSG_OK) return -1;
  int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot)
  for (int64_t k = 0; k < c.nk; ++k) {
    counts[k] = layer_count(&c, k);
    tot += counts[k];
  }
  needle_free(&c);
  return tot;
}

/* fill layers [k0, k1) contiguously into xyz/type/dsrf; counts from psg_needle_plan */
int psg_needle_fill(const psg_needle_t* p, int64_t k0, int64_t k1, const int64_t* counts, float* xyz,
                    uint8_t* type, float* dsrf) {
  needle_ctx c;
  int rc = needle_init(&c, p);
  if (rc != PSG_OK) return rc;
  if (k0 < 0 || k1 > c.nk || k0 > k1) {
    needle_free(&c);
    return PSG_ERR_ARG;
  }
  int64_t* off = (int64_t*)malloc((size_t)(k1 - k0 + 1) * sizeof(int64_t));
  if (!off) {
    needle_free(&c);
    return PSG_ERR_OOM;
  }
  off[0] = 0;
  for (int64_t k = k0; k < k1; ++k) off[k - k0 + 1] = off[k - k0] + counts[k];
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t o = off[k - k0];
    layer_fill(&c, k, xyz + 3 * o, type + o, dsrf + o);
  }
  free(off);
  needle_free(&c);
  return PSG_OK;
}

/* number of precipitates whose centre lies inside the frustum (for reporting) */
int64_t psg_needle_precipitates(const psg_needle_t* p) {
  needle_ctx c;
  if (needle_init(&c, p) != PSG_OK) return -1;
  int64_t n = 0;
  const int64_t nb = c.nbx * c.nby * c.nbz;
  for (int64_t m = 0; m < c.blk_off[nb]; ++m) {
    const double x = c.prec[4 * m], y = c.prec[4 * m + 1], z = c.prec[4 * m + 2];
    if (z < 0 || z >= p->height) continue;
    const double R = c.rb - z * c.tana;
    if (x * x + y * y < R * R) ++n;
  }
  needle_free(&c);
  return n;
}

int psg_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
