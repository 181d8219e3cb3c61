/*
 * ORACLE for the spatial-statistics hot path.  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg may call
 * it; the product path never does.  It shares no code with the CUDA path.
 *
 * Plain, slow, single-threaded C.  Every function is the definition written
 * out, following the paper:
 *   - kNN: distribution of the distance from each central ion of the chosen
 *     types to its k-th nearest neighbour of the chosen types
 *     (Methods, "Descriptive, two-point spatial statistics, and clustering";
 *     Suppl. Fig. SchematicKNN).
 *   - RDF: number of neighbours of the chosen types in radial shells about
 *     each central ion (same passages; Suppl. Fig. SchematicRDF), binned with
 *     rectangular transfer functions on r = [start, step, stop].
 *   - central ions are only those whose distance to the specimen edge is at
 *     least d_srf (Methods, "Quantification of the edge of the point cloud",
 *     "Ion-to-edge distancing"); neighbours are not filtered.
 *   - one spherical ROI about every central ion (Suppl., "Customized user
 *     defined batch processing queues").
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - squared distance in float32, d2 = ((dx*dx)+(dy*dy))+(dz*dz), every
 *     operation rounded to nearest, no contraction (compile with
 *     -ffp-contract=off), dx = x_j - x_i;
 *   - bin edges E[b] = (float)(e_b*e_b), e_b = r0 + b*dr in double, and a pair
 *     lies in bin b when E[b] <= d2 < E[b+1] (half-open in squared distance);
 *   - the self pair is excluded by index, never by distance;
 *   - the kNN search set of ion i is every neighbour j != i with d2 < E[n];
 *     fewer than k of them is "not found";
 *   - smoothed RDF: each pair spreads a Gaussian of width sigma, integrated
 *     over every bin (the rectangular transfer function convolved with a
 *     Gaussian), over the pairs with s*d < stop + 6 sigma;
 *   - spatial distribution map: the pairs with d2 < (float)(R*R) binned by
 *     their float32 displacement x_j - x_i into cubic voxels, edges
 *     V[m] = (float)((m - n_vox/2) * w), half-open on every axis;
 *   - maximum-separation clustering: ions linked when d2 <= (float)(d_max^2)
 *     (closed, as the eps-neighbourhood of DBScan), clusters = connected
 *     components with >= N_min ions, labelled by their smallest ion index.
 *
 * Status codes: 0 ok, 1 bad argument, 2 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2

static int in_mask(const uint64_t* m, uint8_t t) { return (int)((m[t >> 6] >> (t & 63)) & 1u); }

/* Bin edges in squared distance. */
void orc_edges(double r0, double dr, uint32_t n_bins, float* E) {
  for (uint32_t b = 0; b <= n_bins; ++b) {
    const double e = r0 + (double)b * dr;
    E[b] = (float)(e * e);
  }
}

/* float32 squared distance, fixed evaluation order */
static float dist2(const float* xi, const float* xj) {
  const float dx = xj[0] - xi[0];
  const float dy = xj[1] - xi[1];
  const float dz = xj[2] - xi[2];
  const float sx = dx * dx;
  const float sy = dy * dy;
  const float sz = dz * dz;
  const float sxy = sx + sy;
  return sxy + sz;
}

/* bin index: the b in [0, n) with E[b] <= d2 < E[b+1]; caller guarantees E[0] <= d2 < E[n] */
static uint32_t bin_of(const float* E, uint32_t n, float d2) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (d2 >= E[mid])
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static int cmp_float(const void* a, const void* b) {
  const float x = *(const float*)a, y = *(const float*)b;
  return (x > y) - (x < y);
}

typedef struct {
  float* v;
  int64_t n, cap;
} flist;

static int flist_push(flist* l, float x) {
  if (l->n == l->cap) {
    int64_t c = l->cap ? 2 * l->cap : 1024;
    float* p = (float*)realloc(l->v, (size_t)c * sizeof(float));
    if (!p) return ORC_ERR_OOM;
    l->v = p;
    l->cap = c;
  }
  l->v[l->n++] = x;
  return ORC_OK;
}

/* Accumulate one central ion from the full list of its in-range squared
 * distances (d2 < E[n], self excluded). */
static void account_central(int64_t i, int64_t n_ions, flist* L, const float* E, uint32_t n_bins,
                            const uint32_t* ks, uint32_t n_k, uint64_t* rdf, uint64_t* rdf_meta, uint64_t* knn,
                            uint64_t* knn_meta, float* kth_d2, uint32_t* n_within) {
  rdf_meta[0] += 1;
  for (int64_t t = 0; t < L->n; ++t) {
    if (L->v[t] < E[0]) {
      rdf_meta[2] += 1;
    } else {
      rdf[bin_of(E, n_bins, L->v[t])] += 1;
      rdf_meta[1] += 1;
    }
  }
  if (n_within) n_within[i] = (uint32_t)L->n;
  if (n_k == 0) return;
  qsort(L->v, (size_t)L->n, sizeof(float), cmp_float);
  for (uint32_t q = 0; q < n_k; ++q) {
    const int64_t k = ks[q];
    if (L->n < k) {
      knn_meta[2 * q + 0] += 1; /* not found */
      if (kth_d2) kth_d2[(int64_t)q * n_ions + i] = INFINITY;
      continue;
    }
    const float dk = L->v[k - 1];
    if (kth_d2) kth_d2[(int64_t)q * n_ions + i] = dk;
    if (dk < E[0])
      knn_meta[2 * q + 1] += 1; /* below the first edge */
    else
      knn[(int64_t)q * n_bins + bin_of(E, n_bins, dk)] += 1;
  }
}

static int check_common(int64_t n, double r0, double dr, uint32_t n_bins, const uint32_t* ks, uint32_t n_k) {
  if (n < 0 || n_bins == 0 || !(dr > 0) || !(r0 >= 0)) return ORC_ERR_ARG;
  for (uint32_t q = 0; q < n_k; ++q)
    if (ks[q] < 1) return ORC_ERR_ARG;
  return ORC_OK;
}

static void zero_outputs(uint32_t n_bins, uint32_t n_k, uint64_t* rdf, uint64_t* rdf_meta, uint64_t* knn,
                         uint64_t* knn_meta) {
  memset(rdf, 0, (size_t)n_bins * sizeof(uint64_t));
  memset(rdf_meta, 0, 3 * sizeof(uint64_t));
  if (n_k) {
    memset(knn, 0, (size_t)n_k * n_bins * sizeof(uint64_t));
    memset(knn_meta, 0, (size_t)n_k * 2 * sizeof(uint64_t));
  }
}

/*
 * Exact kNN and RDF histograms with a cell list (regular binning, Suppl. Fig.
 * QueryingStructures c).  Outputs:
 *   rdf[n_bins], rdf_meta[3] = {n_central, pairs binned, pairs below E[0]}
 *   knn[n_k][n_bins], knn_meta[n_k][2] = {not found, k-th distance below E[0]}
 *   kth_d2[n_k][n] (optional): k-th squared distance of each central, +inf
 *     when not found; entries of non-central ions are left untouched
 *   n_within[n] (optional): in-range neighbour count of each central
 */
int orc_spatstat(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
                 const uint64_t* nbr_mask, float dsrf_min, double r0, double dr, uint32_t n_bins, const uint32_t* ks,
                 uint32_t n_k, uint64_t* rdf, uint64_t* rdf_meta, uint64_t* knn, uint64_t* knn_meta, float* kth_d2,
                 uint32_t* n_within) {
  int rc = check_common(n, r0, dr, n_bins, ks, n_k);
  if (rc) return rc;
  zero_outputs(n_bins, n_k, rdf, rdf_meta, knn, knn_meta);
  float* E = (float*)malloc((size_t)(n_bins + 1) * sizeof(float));
  if (!E) return ORC_ERR_OOM;
  orc_edges(r0, dr, n_bins, E);
  /* cell edge: a margin above the search radius so every in-range pair lies in adjacent cells */
  const double rs = sqrt((double)E[n_bins]);
  const double h = rs * (1.0 + 1e-5) + 1e-6;

  /* neighbour list by cell: bounding box of the neighbour set */
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int64_t nn = 0;
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    ++nn;
    for (int a = 0; a < 3; ++a) {
      if (xyz[3 * j + a] < lo[a]) lo[a] = xyz[3 * j + a];
      if (xyz[3 * j + a] > hi[a]) hi[a] = xyz[3 * j + a];
    }
  }
  int64_t dim[3] = {1, 1, 1};
  if (nn > 0)
    for (int a = 0; a < 3; ++a) dim[a] = (int64_t)floor((hi[a] - lo[a]) / h) + 1;
  else
    lo[0] = lo[1] = lo[2] = 0.0;
  const int64_t ncell = dim[0] * dim[1] * dim[2];
  int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t* item = (int64_t*)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc((size_t)ncell, sizeof(int64_t));
  flist L = {0, 0, 0};
  if (!start || !item || !fill) {
    rc = ORC_ERR_OOM;
    goto done;
  }
#define CELLC(x, a) ((int64_t)fmin(fmax(floor(((double)(x) - lo[a]) / h), 0.0), (double)(dim[a] - 1)))
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    const int64_t c = (CELLC(xyz[3 * j + 2], 2) * dim[1] + CELLC(xyz[3 * j + 1], 1)) * dim[0] + CELLC(xyz[3 * j], 0);
    start[c + 1] += 1;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    const int64_t c = (CELLC(xyz[3 * j + 2], 2) * dim[1] + CELLC(xyz[3 * j + 1], 1)) * dim[0] + CELLC(xyz[3 * j], 0);
    item[start[c] + fill[c]++] = j;
  }

  for (int64_t i = 0; i < n; ++i) {
    if (!in_mask(ctr_mask, type[i]) || !(dsrf[i] >= dsrf_min)) continue;
    const float* xi = xyz + 3 * i;
    const int64_t cx = CELLC(xi[0], 0), cy = CELLC(xi[1], 1), cz = CELLC(xi[2], 2);
    L.n = 0;
    for (int64_t z = cz - 1; z <= cz + 1; ++z)
      for (int64_t y = cy - 1; y <= cy + 1; ++y)
        for (int64_t x = cx - 1; x <= cx + 1; ++x) {
          if (x < 0 || y < 0 || z < 0 || x >= dim[0] || y >= dim[1] || z >= dim[2]) continue;
          const int64_t c = (z * dim[1] + y) * dim[0] + x;
          for (int64_t t = start[c]; t < start[c + 1]; ++t) {
            const int64_t j = item[t];
            if (j == i) continue;
            const float d2 = dist2(xi, xyz + 3 * j);
            if (d2 < E[n_bins] && flist_push(&L, d2)) {
              rc = ORC_ERR_OOM;
              goto done;
            }
          }
        }
    account_central(i, n, &L, E, n_bins, ks, n_k, rdf, rdf_meta, knn, knn_meta, kth_d2, n_within);
  }
#undef CELLC
done:
  free(L.v);
  free(fill);
  free(item);
  free(start);
  free(E);
  return rc;
}

/*
 * Normalised RDF g(r) from the integer histogram (a derived output; the
 * paper names the RDF as the distribution of neighbours in radial shells
 * about every central ion, Methods "Descriptive, two-point spatial
 * statistics, and clustering", and gives no normalisation).  Reading: the
 * counts of bin b are divided by what a uniform neighbour density would put
 * in that shell about every central:
 *   g_b = H[b] / (n_central * rho * V_b),  rho = n_nbr / volume,
 *   V_b = 4/3 pi (e_{b+1}^3 - e_b^3),  e_b = r0 + b dr   (double).
 * n_central = 0 or n_nbr = 0 gives g = 0.  FP64.
 */
int orc_rdf_normalise(const uint64_t* rdf, uint32_t n_bins, double r0, double dr, uint64_t n_central,
                      uint64_t n_nbr, double volume, double* g) {
  if (n_bins == 0 || !(dr > 0) || !(r0 >= 0) || !(volume > 0)) return ORC_ERR_ARG;
  const double rho = (double)n_nbr / volume;
  for (uint32_t b = 0; b < n_bins; ++b) {
    const double e0 = r0 + (double)b * dr, e1 = r0 + (double)(b + 1) * dr;
    const double shell = 4.0 / 3.0 * M_PI * (e1 * e1 * e1 - e0 * e0 * e0);
    const double expected = (double)n_central * rho * shell;
    g[b] = expected > 0.0 ? (double)rdf[b] / expected : 0.0;
  }
  return ORC_OK;
}

/* Same contract as orc_spatstat, by O(N^2) brute force (no spatial index). */
int orc_spatstat_brute(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
                       const uint64_t* nbr_mask, float dsrf_min, double r0, double dr, uint32_t n_bins,
                       const uint32_t* ks, uint32_t n_k, uint64_t* rdf, uint64_t* rdf_meta, uint64_t* knn,
                       uint64_t* knn_meta, float* kth_d2, uint32_t* n_within) {
  int rc = check_common(n, r0, dr, n_bins, ks, n_k);
  if (rc) return rc;
  zero_outputs(n_bins, n_k, rdf, rdf_meta, knn, knn_meta);
  float* E = (float*)malloc((size_t)(n_bins + 1) * sizeof(float));
  if (!E) return ORC_ERR_OOM;
  orc_edges(r0, dr, n_bins, E);
  flist L = {0, 0, 0};
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
    if (!in_mask(ctr_mask, type[i]) || !(dsrf[i] >= dsrf_min)) continue;
    L.n = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i || !in_mask(nbr_mask, type[j])) continue;
      const float d2 = dist2(xyz + 3 * i, xyz + 3 * j);
      if (d2 < E[n_bins] && flist_push(&L, d2)) {
        rc = ORC_ERR_OOM;
        break;
      }
    }
    if (rc == ORC_OK)
      account_central(i, n, &L, E, n_bins, ks, n_k, rdf, rdf_meta, knn, knn_meta, kth_d2, n_within);
  }
  free(L.v);
  free(E);
  return rc;
}

/*
 * One central ion i by brute force over all n ions (for sampled checks on
 * clouds too large for the full oracle).  Outputs the in-range neighbour
 * count, the k-th squared distances (kth_d2[n_k], +inf when not found) and,
 * optionally, its own RDF counts (rdf_i[n_bins], may be NULL).
 */
int orc_central_brute(const float* xyz, const uint8_t* type, int64_t n, int64_t i, const uint64_t* nbr_mask,
                      double r0, double dr, uint32_t n_bins, const uint32_t* ks, uint32_t n_k, float* kth_d2,
                      uint32_t* n_within, uint64_t* rdf_i) {
  int rc = check_common(n, r0, dr, n_bins, ks, n_k);
  if (rc) return rc;
  if (i < 0 || i >= n) return ORC_ERR_ARG;
  float* E = (float*)malloc((size_t)(n_bins + 1) * sizeof(float));
  if (!E) return ORC_ERR_OOM;
  orc_edges(r0, dr, n_bins, E);
  flist L = {0, 0, 0};
  for (int64_t j = 0; j < n; ++j) {
    if (j == i || !in_mask(nbr_mask, type[j])) continue;
    const float d2 = dist2(xyz + 3 * i, xyz + 3 * j);
    if (d2 < E[n_bins] && flist_push(&L, d2)) {
      free(L.v);
      free(E);
      return ORC_ERR_OOM;
    }
  }
  *n_within = (uint32_t)L.n;
  if (rdf_i) {
    memset(rdf_i, 0, (size_t)n_bins * sizeof(uint64_t));
    for (int64_t t = 0; t < L.n; ++t)
      if (L.v[t] >= E[0]) rdf_i[bin_of(E, n_bins, L.v[t])] += 1;
  }
  qsort(L.v, (size_t)L.n, sizeof(float), cmp_float);
  for (uint32_t q = 0; q < n_k; ++q) kth_d2[q] = (L.n >= (int64_t)ks[q]) ? L.v[ks[q] - 1] : INFINITY;
  free(L.v);
  free(E);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Spatial distribution map: the three-dimensional two-point statistic of     */
/* which RDF and kNN are annular integrals (Methods, "Descriptive, two-point  */
/* spatial statistics, and clustering"; Results, strong scaling: cubic voxels */
/* about each central ion, ROI radius R).                                     */
/*                                                                            */
/*  for every central i and neighbour j != i with d2_ij < (float)(R*R):        */
/*     the displacement (dx, dy, dz) = x_j - x_i (float32, as for d2) falls    */
/*     in voxel (mx, my, mz) with V[m] <= d < V[m+1] on each axis,             */
/*     V[m] = (float)((m - n_vox/2) * w) in double, m = 0..n_vox;              */
/*     H[(mz*n_vox + my)*n_vox + mx] += 1.  A displacement outside the cube    */
/*     [V[0], V[n_vox])^3 is counted in meta[2] instead.                       */
/*  meta = {n_central, pairs in the map, pairs outside the cube}.             */
/* ------------------------------------------------------------------------- */
void orc_sdm_edges(double w, uint32_t n_vox, float* V) {
  for (uint32_t m = 0; m <= n_vox; ++m) V[m] = (float)(((double)m - (double)n_vox / 2.0) * w);
}

/* voxel index along one axis: the m in [0, n) with V[m] <= d < V[m+1]; -1 outside [V[0], V[n]) */
static int64_t vox_of(const float* V, uint32_t n, float d) {
  if (!(d >= V[0]) || !(d < V[n])) return -1;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (d >= V[mid])
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

int orc_sdm(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
            const uint64_t* nbr_mask, float dsrf_min, double r_max, double w, uint32_t n_vox, uint64_t* H,
            uint64_t* meta) {
  if (n < 0 || !(r_max > 0) || !(w > 0) || n_vox == 0 || n_vox > 1024) return ORC_ERR_ARG;
  const size_t nh = (size_t)n_vox * n_vox * n_vox;
  memset(H, 0, nh * sizeof(uint64_t));
  meta[0] = meta[1] = meta[2] = 0;
  float* V = (float*)malloc((size_t)(n_vox + 1) * sizeof(float));
  if (!V) return ORC_ERR_OOM;
  orc_sdm_edges(w, n_vox, V);
  const float ER = (float)(r_max * r_max);
  /* cell list of the neighbour set, cells of edge just above R */
  const double h = sqrt((double)ER) * (1.0 + 1e-5) + 1e-6;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int64_t nn = 0;
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    ++nn;
    for (int a = 0; a < 3; ++a) {
      if (xyz[3 * j + a] < lo[a]) lo[a] = xyz[3 * j + a];
      if (xyz[3 * j + a] > hi[a]) hi[a] = xyz[3 * j + a];
    }
  }
  int64_t dim[3] = {1, 1, 1};
  if (nn > 0)
    for (int a = 0; a < 3; ++a) dim[a] = (int64_t)floor((hi[a] - lo[a]) / h) + 1;
  else
    lo[0] = lo[1] = lo[2] = 0.0;
  const int64_t ncell = dim[0] * dim[1] * dim[2];
  int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t* item = (int64_t*)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc((size_t)ncell, sizeof(int64_t));
  int rc = ORC_OK;
  if (!start || !item || !fill) {
    rc = ORC_ERR_OOM;
    goto done;
  }
#define CELLS(x, a) ((int64_t)fmin(fmax(floor(((double)(x) - lo[a]) / h), 0.0), (double)(dim[a] - 1)))
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    start[(CELLS(xyz[3 * j + 2], 2) * dim[1] + CELLS(xyz[3 * j + 1], 1)) * dim[0] + CELLS(xyz[3 * j], 0) + 1] += 1;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  for (int64_t j = 0; j < n; ++j) {
    if (!in_mask(nbr_mask, type[j])) continue;
    const int64_t c = (CELLS(xyz[3 * j + 2], 2) * dim[1] + CELLS(xyz[3 * j + 1], 1)) * dim[0] + CELLS(xyz[3 * j], 0);
    item[start[c] + fill[c]++] = j;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!in_mask(ctr_mask, type[i]) || !(dsrf[i] >= dsrf_min)) continue;
    meta[0] += 1;
    const float* xi = xyz + 3 * i;
    const int64_t cx = CELLS(xi[0], 0), cy = CELLS(xi[1], 1), cz = CELLS(xi[2], 2);
    for (int64_t z = cz - 1; z <= cz + 1; ++z)
      for (int64_t y = cy - 1; y <= cy + 1; ++y)
        for (int64_t x = cx - 1; x <= cx + 1; ++x) {
          if (x < 0 || y < 0 || z < 0 || x >= dim[0] || y >= dim[1] || z >= dim[2]) continue;
          const int64_t c = (z * dim[1] + y) * dim[0] + x;
          for (int64_t t = start[c]; t < start[c + 1]; ++t) {
            const int64_t j = item[t];
            if (j == i) continue;
            const float* xj = xyz + 3 * j;
            if (!(dist2(xi, xj) < ER)) continue;
            const int64_t mx = vox_of(V, n_vox, xj[0] - xi[0]);
            const int64_t my = vox_of(V, n_vox, xj[1] - xi[1]);
            const int64_t mz = vox_of(V, n_vox, xj[2] - xi[2]);
            if (mx < 0 || my < 0 || mz < 0) {
              meta[2] += 1;
            } else {
              H[((size_t)mz * n_vox + (size_t)my) * n_vox + (size_t)mx] += 1;
              meta[1] += 1;
            }
          }
        }
  }
#undef CELLS
done:
  free(fill);
  free(item);
  free(start);
  free(V);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Maximum-separation clustering (Methods, "Descriptive, two-point spatial    */
/* statistics, and clustering": the DBScan variant with the threshold          */
/* distance d_max and the minimum cluster size N_min; Results on the AM        */
/* specimens for the post-processing of the labels).                          */
/*                                                                            */
/*  Ions of the chosen types are linked when d2 <= (float)(d_max^2) (float32  */
/*  d2 as everywhere); clusters are the connected components with at least    */
/*  n_min ions.  Outputs:                                                     */
/*   label[n]  smallest original index in the ion's cluster, or 0xFFFFFFFF     */
/*             (other types, or a component smaller than n_min)               */
/*   size_hist[hist_len]  clusters by size (sizes >= hist_len-1 in the last    */
/*             entry); interior_hist likewise for the clusters whose members  */
/*             all have d_srf >= dsrf_min (not truncated by the edge)         */
/*   meta = {n_set, n_clusters, ions in clusters, interior clusters}          */
/* ------------------------------------------------------------------------- */
static int64_t uf_find(int64_t* parent, int64_t x) {
  while (parent[x] != x) x = parent[x];
  return x;
}

int orc_cluster(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* mask,
                double d_max, uint32_t n_min, float dsrf_min, uint32_t hist_len, uint32_t* label,
                uint64_t* size_hist, uint64_t* interior_hist, uint64_t* meta) {
  if (n < 0 || !(d_max > 0) || n_min < 1 || hist_len < 2) return ORC_ERR_ARG;
  const float D = (float)(d_max * d_max);
  memset(size_hist, 0, (size_t)hist_len * sizeof(uint64_t));
  memset(interior_hist, 0, (size_t)hist_len * sizeof(uint64_t));
  meta[0] = meta[1] = meta[2] = meta[3] = 0;
  for (int64_t i = 0; i < n; ++i) label[i] = 0xFFFFFFFFu;
  int64_t* parent = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* csize = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t* cmin = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  float* cdmin = (float*)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
  int64_t* start = NULL;
  int64_t* item = NULL;
  int64_t* fill = NULL;
  int rc = ORC_OK;
  if (!parent || !csize || !cmin || !cdmin) {
    rc = ORC_ERR_OOM;
    goto done;
  }
  for (int64_t i = 0; i < n; ++i) parent[i] = i;
  /* cell list of the set, cells of edge just above d_max */
  {
    const double h = sqrt((double)D) * (1.0 + 1e-5) + 1e-6;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int64_t nn = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (!in_mask(mask, type[j])) continue;
      ++nn;
      for (int a = 0; a < 3; ++a) {
        if (xyz[3 * j + a] < lo[a]) lo[a] = xyz[3 * j + a];
        if (xyz[3 * j + a] > hi[a]) hi[a] = xyz[3 * j + a];
      }
    }
    meta[0] = (uint64_t)nn;
    int64_t dim[3] = {1, 1, 1};
    if (nn > 0)
      for (int a = 0; a < 3; ++a) dim[a] = (int64_t)floor((hi[a] - lo[a]) / h) + 1;
    else
      lo[0] = lo[1] = lo[2] = 0.0;
    const int64_t ncell = dim[0] * dim[1] * dim[2];
    start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    item = (int64_t*)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int64_t));
    fill = (int64_t*)calloc((size_t)ncell, sizeof(int64_t));
    if (!start || !item || !fill) {
      rc = ORC_ERR_OOM;
      goto done;
    }
#define CELLK(x, a) ((int64_t)fmin(fmax(floor(((double)(x) - lo[a]) / h), 0.0), (double)(dim[a] - 1)))
    for (int64_t j = 0; j < n; ++j) {
      if (!in_mask(mask, type[j])) continue;
      start[(CELLK(xyz[3 * j + 2], 2) * dim[1] + CELLK(xyz[3 * j + 1], 1)) * dim[0] + CELLK(xyz[3 * j], 0) + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t j = 0; j < n; ++j) {
      if (!in_mask(mask, type[j])) continue;
      const int64_t c = (CELLK(xyz[3 * j + 2], 2) * dim[1] + CELLK(xyz[3 * j + 1], 1)) * dim[0] + CELLK(xyz[3 * j], 0);
      item[start[c] + fill[c]++] = j;
    }
    /* link every pair within d_max: union of the two components (larger root under the smaller) */
    for (int64_t i = 0; i < n; ++i) {
      if (!in_mask(mask, type[i])) continue;
      const float* xi = xyz + 3 * i;
      const int64_t cx = CELLK(xi[0], 0), cy = CELLK(xi[1], 1), cz = CELLK(xi[2], 2);
      for (int64_t z = cz - 1; z <= cz + 1; ++z)
        for (int64_t y = cy - 1; y <= cy + 1; ++y)
          for (int64_t x = cx - 1; x <= cx + 1; ++x) {
            if (x < 0 || y < 0 || z < 0 || x >= dim[0] || y >= dim[1] || z >= dim[2]) continue;
            const int64_t c = (z * dim[1] + y) * dim[0] + x;
            for (int64_t t = start[c]; t < start[c + 1]; ++t) {
              const int64_t j = item[t];
              if (j <= i || !(dist2(xi, xyz + 3 * j) <= D)) continue;
              const int64_t ri = uf_find(parent, i), rj = uf_find(parent, j);
              if (ri < rj)
                parent[rj] = ri;
              else if (rj < ri)
                parent[ri] = rj;
            }
          }
    }
#undef CELLK
  }
  /* components: the root is the smallest index of the component */
  for (int64_t i = 0; i < n; ++i) {
    cmin[i] = -1;
    cdmin[i] = INFINITY;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!in_mask(mask, type[i])) continue;
    const int64_t r = uf_find(parent, i);
    csize[r] += 1;
    if (cmin[r] < 0 || i < cmin[r]) cmin[r] = i;
    if (dsrf[i] < cdmin[r]) cdmin[r] = dsrf[i];
  }
  for (int64_t r = 0; r < n; ++r) {
    if (csize[r] < (int64_t)n_min) continue;
    const uint32_t b = csize[r] >= (int64_t)hist_len - 1 ? hist_len - 1 : (uint32_t)csize[r];
    size_hist[b] += 1;
    meta[1] += 1;
    meta[2] += (uint64_t)csize[r];
    if (cdmin[r] >= dsrf_min) {
      interior_hist[b] += 1;
      meta[3] += 1;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!in_mask(mask, type[i])) continue;
    const int64_t r = uf_find(parent, i);
    if (csize[r] >= (int64_t)n_min) label[i] = (uint32_t)cmin[r];
  }
done:
  free(fill);
  free(item);
  free(start);
  free(cdmin);
  free(cmin);
  free(csize);
  free(parent);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Gaussian-smoothed RDF and its adjoint, in FP64.                            */
/*                                                                            */
/*  u_ij = s * |x_j - x_i|  (FP64 from the float32 coordinates)               */
/*  h[b] = sum over central i, neighbour j != i with u_ij < stop + 6 sigma of */
/*         Phi((e_{b+1} - u_ij)/sigma) - Phi((e_b - u_ij)/sigma)              */
/*  Given G[b] = dL/dh[b], the adjoint of every pair is                       */
/*     w_ij = sum_b G[b] (phi((e_b - u)/sigma) - phi((e_{b+1} - u)/sigma))/sigma */
/*  = dL/du_ij, and du/dx_i = s (x_i - x_j)/d, du/dx_j = -du/dx_i, du/ds = d. */
/* ------------------------------------------------------------------------- */
static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }
static double phi(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * M_PI); }

static int soft_pairs(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
                      const uint64_t* nbr_mask, float dsrf_min, double sigma, double scale, double r0, double dr,
                      uint32_t n_bins, const double* G, double* h, double* grad_xyz, double* grad_s) {
  if (n < 0 || n_bins == 0 || !(dr > 0) || !(r0 >= 0) || !(sigma > 0) || !(scale > 0)) return ORC_ERR_ARG;
  const double rcut = r0 + (double)n_bins * dr + 6.0 * sigma;
  double* e = (double*)malloc((size_t)(n_bins + 1) * sizeof(double));
  if (!e) return ORC_ERR_OOM;
  for (uint32_t b = 0; b <= n_bins; ++b) e[b] = r0 + (double)b * dr;
  double* P = (double*)malloc((size_t)(n_bins + 1) * sizeof(double));
  if (!P) {
    free(e);
    return ORC_ERR_OOM;
  }
  if (h) memset(h, 0, (size_t)n_bins * sizeof(double));
  if (grad_xyz) memset(grad_xyz, 0, (size_t)n * 3 * sizeof(double));
  if (grad_s) *grad_s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!in_mask(ctr_mask, type[i]) || !(dsrf[i] >= dsrf_min)) continue;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i || !in_mask(nbr_mask, type[j])) continue;
      const double v0 = (double)xyz[3 * i + 0] - (double)xyz[3 * j + 0];
      const double v1 = (double)xyz[3 * i + 1] - (double)xyz[3 * j + 1];
      const double v2 = (double)xyz[3 * i + 2] - (double)xyz[3 * j + 2];
      const double d = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      const double u = scale * d;
      if (!(u < rcut)) continue;
      if (h) {
        for (uint32_t b = 0; b <= n_bins; ++b) P[b] = Phi((e[b] - u) / sigma);
        for (uint32_t b = 0; b < n_bins; ++b) h[b] += P[b + 1] - P[b];
      }
      if (G) {
        double w = 0.0;
        for (uint32_t b = 0; b < n_bins; ++b) w += G[b] * (phi((e[b] - u) / sigma) - phi((e[b + 1] - u) / sigma)) / sigma;
        if (grad_s) *grad_s += w * d;
        if (grad_xyz && d > 0.0) {
          const double f = w * scale / d;
          grad_xyz[3 * i + 0] += f * v0;
          grad_xyz[3 * i + 1] += f * v1;
          grad_xyz[3 * i + 2] += f * v2;
          grad_xyz[3 * j + 0] -= f * v0;
          grad_xyz[3 * j + 1] -= f * v1;
          grad_xyz[3 * j + 2] -= f * v2;
        }
      }
    }
  }
  free(P);
  free(e);
  return ORC_OK;
}

int orc_soft_fwd(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
                 const uint64_t* nbr_mask, float dsrf_min, double sigma, double scale, double r0, double dr,
                 uint32_t n_bins, double* h) {
  return soft_pairs(xyz, type, dsrf, n, ctr_mask, nbr_mask, dsrf_min, sigma, scale, r0, dr, n_bins, NULL, h, NULL,
                    NULL);
}

int orc_soft_bwd(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n, const uint64_t* ctr_mask,
                 const uint64_t* nbr_mask, float dsrf_min, double sigma, double scale, double r0, double dr,
                 uint32_t n_bins, const double* G, double* grad_xyz, double* grad_s) {
  if (!G) return ORC_ERR_ARG;
  return soft_pairs(xyz, type, dsrf, n, ctr_mask, nbr_mask, dsrf_min, sigma, scale, r0, dr, n_bins, G, NULL,
                    grad_xyz, grad_s);
}

/* ------------------------------------------------------------------------- */
/* Randomised type labels (Suppl. "Importance of high quality random number   */
/* generators": every statistic is also computed for a random relabelling).   */
/*                                                                            */
/* The relabelling is out[i] = in[perm(i)] with perm a pseudo-random          */
/* permutation of [0, n): a 4-round Feistel network over 2h bits              */
/* (2^(2h) >= n, h >= 1) whose round function is the splitmix64 finaliser of  */
/* (half-block + round key), round key r = finaliser(seed + (r + 1) * golden  */
/* gamma), restricted to [0, n) by cycle walking (apply the network again      */
/* until the value falls below n).                                            */
/* ------------------------------------------------------------------------- */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t feistel(uint64_t x, const uint64_t key[4], unsigned h) {
  const uint64_t mask = (h >= 64) ? ~0ULL : ((1ULL << h) - 1);
  uint64_t L = x >> h, R = x & mask;
  for (int r = 0; r < 4; ++r) {
    const uint64_t t = L ^ (sm64_mix(R + key[r]) & mask);
    L = R;
    R = t;
  }
  return (L << h) | R;
}

void orc_label_perm(int64_t n, uint64_t seed, uint32_t* perm) {
  unsigned h = 1;
  while ((1ULL << (2 * h)) < (uint64_t)n) ++h;
  uint64_t key[4];
  for (int r = 0; r < 4; ++r) key[r] = sm64_mix(seed + (uint64_t)(r + 1) * 0x9e3779b97f4a7c15ULL);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t y = feistel((uint64_t)i, key, h);
    while (y >= (uint64_t)n) y = feistel(y, key, h);
    perm[i] = (uint32_t)y;
  }
}

int orc_shuffle_labels(const uint8_t* in, uint8_t* out, int64_t n, uint64_t seed) {
  if (n < 0 || n > 0xFFFFFFFFLL) return ORC_ERR_ARG;
  uint32_t* perm = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
  if (!perm) return ORC_ERR_OOM;
  orc_label_perm(n, seed, perm);
  for (int64_t i = 0; i < n; ++i) out[i] = in[perm[i]];
  free(perm);
  return ORC_OK;
}
