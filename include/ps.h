/*
 * ps.h — C ABI of libps: exact kNN / RDF spatial statistics of atom-probe
 * point clouds on one GB300 (sm_103a), plus the batched sweep and the
 * Gaussian-smoothed RDF with its adjoint.
 *
 * What is computed (the paper's spatial-statistics task, Methods
 * "Descriptive, two-point spatial statistics, and clustering"; Suppl.
 * "Efficient batch processing of spatial statistics", Figs. SchematicKNN and
 * SchematicRDF):
 *   central set   C = { i : type_i in ctr_mask and d_srf_i >= dsrf_min }
 *                 (the d_srf edge rule of Methods "Ion-to-edge distancing";
 *                 neighbours are never d_srf-filtered)
 *   neighbour set N = { j : type_j in nbr_mask }
 *   d2_ij         = ((dx*dx)+(dy*dy))+(dz*dz) in float32, dx = x_j - x_i,
 *                 every operation rounded to nearest, no FMA contraction
 *   edges         E[b] = (float)((r0 + b*dr)^2), r0 and dr double, b = 0..n_bins
 *                 (the paper's bin notation r = [start, step, stop], with
 *                 n_bins = round((stop - start)/step))
 *   RDF           H[b] = #{ (i, j) : i in C, j in N, j != i, E[b] <= d2_ij < E[b+1] }
 *                 (ordered pairs; the self pair is excluded by index)
 *   kNN           D_k(i) = k-th smallest d2_ij over j in N, j != i,
 *                 d2_ij < E[n_bins]; K[b] counts the centrals whose D_k falls in
 *                 bin b; fewer than k such j is "not found".
 * All histograms are exact integers, bit-identical to the definition.
 *
 * Conventions for every entry point:
 *   - Arrays named d_* and the xyz/type/dsrf inputs are DEVICE pointers
 *     owned by the caller.  xyz is float32 [n][3] (x, y, z interleaved, nm),
 *     type is uint8 [n], dsrf is float32 [n].  Inputs are read only; they
 *     must stay valid and unchanged while any call that uses them (or a
 *     grid built from them) is in flight.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously; results are valid once the
 *     stream reaches that point.  Unless stated, no call synchronises.
 *   - Type sets are uint64_t[4] bit masks over the 256 possible labels
 *     (bit t of word t/64 set = label t in the set).
 *   - Every function returns a ps_status.  Errors found on the host return
 *     immediately with nothing enqueued; ps_last_error() (thread local)
 *     describes the last failure.  Errors found on the device (non-finite
 *     coordinates, a bounded wait that timed out) are written to the status
 *     word of the output meta array (index PS_META_STATUS) and to the grid's
 *     status, read with ps_grid_get_info().  No call aborts the process, traps
 *     the GPU or throws across the ABI.
 *   - Output histograms and meta arrays are overwritten, not accumulated.
 *   - Limits: n < 2^32 ions; 1 <= n_bins <= PS_MAX_BINS; 1 <= k <= PS_K_MAX.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PS_API __attribute__((visibility("default")))
#else
#define PS_API
#endif

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter (host check) */
  PS_ERR_INVALID_INPUT = 2, /* non-finite coordinate found on the device */
  PS_ERR_OOM = 3,           /* device allocation failed */
  PS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  PS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  PS_ERR_UNSUPPORTED = 6,   /* k > PS_K_MAX, too many bins, ... */
  PS_ERR_CAPACITY = 7       /* n larger than the grid was created for */
} ps_status;

#define PS_K_MAX 32
#define PS_MAX_BINS 8192
#define PS_MAX_KLIST 32

/* Layout of the uint64 meta array written by the histogram calls. */
#define PS_META_N_CENTRAL 0 /* |C| */
#define PS_META_N_PAIRS 1   /* RDF pairs binned (sum of H) */
#define PS_META_N_BELOW 2   /* RDF pairs with d2 < E[0] (only when r0 > 0) */
#define PS_META_STATUS 3    /* 0, or the ps_status of a device-side error */
#define PS_META_HEAD 4
/* then, for the q-th requested k: [PS_META_HEAD + 2q] not found,
 * [PS_META_HEAD + 2q + 1] k-th distance below E[0] */
#define PS_META_LEN(n_k) (PS_META_HEAD + 2 * (n_k))

/* Bins r = [r0, r0 + n_bins*dr) in nm; see the edge rule above. */
typedef struct {
  double r0;
  double dr;
  uint32_t n_bins;
} ps_bins;

/* Options for a cell grid.  struct_size = sizeof(ps_grid_opts). */
typedef struct {
  uint32_t struct_size;
  float cell_scale;   /* cell edge = r_cut * cell_scale; 0 = default (1.0).  >= 1: the 27 cells
                         around a cell are searched; in [0.5, 1): the 125 cells within two cells;
                         in [1/3, 0.5): the 343 cells within three cells.  Cells that cannot hold
                         a record within r_cut of the cell (their gap to it exceeds r_cut on the
                         cell-edge lower bound) are skipped by the exact query: the 4 far corner
                         cells of each octant (32 of 343) for 1/3.  Below 1/3:
                         PS_ERR_INVALID_ARG */
  uint32_t block;     /* reserved (0) */
  uint32_t dense_min; /* cells with at least this many centrals use the CTA kernel that stages the
                         neighbour cells in shared memory with bulk copies; 0 = never */
  uint32_t split;     /* 1: with cell_scale < 1, an exact query that wants the RDF and no per-central
                         in-range counts, and central types among the neighbour types, runs in passes:
                         kNN near each central (cell_scale >= 0.5: the 2 x 2 x 2 cells around its
                         nearest grid vertex, within its distance to their faces; below 0.5: the 27
                         cells around its cell) with a full-radius search only for the centrals that
                         have fewer than k neighbours there, and the RDF over unordered pairs (each
                         pair tested once, counted once per central end).  Same results; 0
                         (default): one combined pass */
} ps_grid_opts;

typedef struct ps_grid ps_grid; /* opaque; owns its device scratch */

/* Library version (major*10000 + minor*100 + patch). */
PS_API int ps_version(void);

/* Description of the last error on this thread ("" if none). */
PS_API const char* ps_last_error(void);

/* Host helper: the edge table E[0..n_bins] (float32, host memory) used by
 * every kernel, by the formula above.  Returns PS_ERR_INVALID_ARG for
 * dr <= 0, r0 < 0, n_bins out of range or E == NULL. */
PS_API int ps_bin_edges(ps_bins bins, float* E);

/*
 * Cell grid over the neighbour set (regular spatial binning, Suppl. Fig.
 * QueryingStructures c, which replaces the paper's per-region KD-trees).
 *
 * ps_grid_create allocates the device scratch for up to n_max ions
 * (about 60 bytes per ion plus the cell arrays); it synchronises the device
 * (cudaMalloc).  ps_grid_build bins the ions j with type_j in nbr_mask into
 * cells of edge >= r_cut, sorted by cell (counting sort), asynchronously on
 * `stream`, with no host synchronisation: the bounding box and the cell
 * dimensions stay on the device.  The grid keeps the xyz and type pointers;
 * later queries read them again.  Returns PS_ERR_CAPACITY if n > n_max,
 * PS_ERR_INVALID_ARG for r_cut <= 0 or null pointers (n == 0 is allowed).
 * ps_build_grid = ps_grid_create(n) + ps_grid_build.
 * ps_grid_destroy frees everything (synchronises; NULL is allowed).
 */
PS_API int ps_grid_create(int64_t n_max, const ps_grid_opts* opts, ps_grid** out);
PS_API int ps_grid_build(ps_grid* g, const float* xyz, const uint8_t* type, int64_t n, const uint64_t nbr_mask[4],
                  float r_cut, void* stream);
PS_API int ps_build_grid(const float* xyz, const uint8_t* type, int64_t n, const uint64_t nbr_mask[4], float r_cut,
                  const ps_grid_opts* opts, void* stream, ps_grid** out);
PS_API int ps_grid_destroy(ps_grid* g);
/* The query options of a grid (ps_grid_opts.dense_min and .split) for its next queries; the cell
 * size stays.  Host only: takes effect for calls enqueued afterwards. */
PS_API int ps_grid_set_query_opts(ps_grid* g, uint32_t dense_min, uint32_t split);

/* Grid geometry, read back from the device (synchronises `stream`). */
typedef struct {
  uint32_t struct_size;
  uint32_t dims[3];
  float origin[3];
  float cell;        /* cell edge (nm) */
  int64_t n_nbr;     /* ions in the neighbour set */
  int64_t n_cells;
  int32_t status;    /* device-side ps_status of the last build */
} ps_grid_info;
PS_API int ps_grid_get_info(ps_grid* g, ps_grid_info* info, void* stream);

/*
 * Exact kNN + RDF in one enumeration of the ROIs.  As in the paper's batch
 * queue (Suppl. "Customized user defined batch processing queues"), the
 * neighbours of a ROI are found once and every requested statistic (each k
 * and the RDF) is evaluated from that one pass.
 *   g         grid built with r_cut >= sqrt(E[n_bins]) (else PS_ERR_INVALID_ARG)
 *   dsrf      device float32 [n] of the grid's cloud; NULL = no d_srf filter
 *   ctr_mask  central types; dsrf_min the d_srf threshold (inclusive)
 *   ks, n_k   HOST array of k values (1..PS_K_MAX), n_k <= PS_MAX_KLIST; n_k may be 0
 *   d_rdf     uint64 [n_bins] or NULL (no RDF)
 *   d_knn     uint64 [n_k][n_bins] or NULL when n_k == 0
 *   d_meta    uint64 [PS_META_LEN(n_k)] (required)
 *   d_kth     optional float32 [n_k][n]: D_k(i) as a squared distance, +inf
 *             when not found; written for central ions only
 *   d_nwithin optional uint32 [n]: in-range neighbours of each central
 *             (d2 < E[n_bins]); written for central ions only
 */
PS_API int ps_spatstat(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
                const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn, uint64_t* d_meta, float* d_kth,
                uint32_t* d_nwithin, void* stream);

/* kNN histogram for one k: ps_spatstat with n_k = 1 and no RDF.
 * d_meta is uint64 [PS_META_LEN(1)]; d_kth optional float32 [n]. */
PS_API int ps_knn_hist(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, uint32_t k,
                ps_bins bins, uint64_t* d_hist, uint64_t* d_meta, float* d_kth, void* stream);

/* RDF histogram: ps_spatstat with n_k = 0.  d_meta is uint64 [PS_META_LEN(0)]. */
PS_API int ps_rdf_hist(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
                uint64_t* d_hist, uint64_t* d_meta, void* stream);

/*
 * Normalised RDF g(r) from the integer histogram (the finalisation step).  The
 * paper reports RDFs normalised (Methods, "Descriptive, two-point spatial
 * statistics, and clustering") without a formula; the reading used here
 * divides each bin by the count a uniform neighbour density rho = |N| / volume
 * puts in that shell about each central:
 *   g_b = H[b] / (|C| * rho * 4/3 pi (e_{b+1}^3 - e_b^3)),  e_b = r0 + b*dr,
 * in FP64 (|C| = 0 or |N| = 0 gives 0).
 *   g        the grid the histogram was computed on, not rebuilt since: |N| is
 *            its neighbour count, read on the device
 *   d_meta   device uint64 meta array of that ps_spatstat / ps_rdf_hist call
 *            (|C| = d_meta[PS_META_N_CENTRAL])
 *   d_rdf    device uint64 [n_bins], the histogram (may be NULL when d_g is)
 *   volume   specimen volume in nm^3 (> 0), the same units as the coordinates
 *   d_g      device double [n_bins] or NULL: g_b
 *   d_factor device double [n_bins] or NULL: 1 / (|C| rho 4/3 pi (e_{b+1}^3 -
 *            e_b^3)), the factor that turns counts (or a smoothed histogram)
 *            into g
 * At least one of d_g and d_factor is required.  Asynchronous on `stream`.
 */
PS_API int ps_rdf_normalise(ps_grid* g, const uint64_t* d_meta, const uint64_t* d_rdf, double volume, ps_bins bins,
                            double* d_g, double* d_factor, void* stream);

/*
 * Batched sweeps over many ROIs in one persistent launch.  The paper's batch
 * queue evaluates an a-priori list of (statistic, type combination, dataset)
 * tasks from one neighbour search per ROI (Suppl. "Customized user defined
 * batch processing queues"); here every ROI is enumerated once at the largest
 * r_max, and each sweep point is derived exactly: all k = 1..k_max from one
 * top-k list, smaller r_max as prefixes of the histograms, d_srf thresholds
 * as sums over d_srf classes, all type pairs from the same enumeration.
 *
 * ps_dataset: one ROI, device pointers (xyz float32 [n][3], type uint8 [n],
 *   dsrf float32 [n] or NULL), n < 2^24 ions; arrays must stay valid while the
 *   batch exists.
 * ps_sweep: the histogram bins at the largest r_max (n_bins <= 512); rmax_bins
 *   the r_max values as ascending bin counts (last = bins.n_bins); dsrf_min the
 *   ascending d_srf thresholds; type pairs (ctr_mask, nbr_mask), at most two
 *   distinct neighbour sets; k = 1..k_max; cell_scale as in ps_grid_opts, 0 or >= 0.5
 *   (PS_ERR_UNSUPPORTED below).
 *   Limit: n_pairs * n_dsrf * n_bins <= 8192.
 * ps_batch_create allocates every grid and accumulator (synchronises).
 * ps_batch_run enqueues the builds of all ROIs, the one persistent query
 *   kernel and the expansion into d_out (uint64, ps_batch_out_len elements):
 *   for each (ROI, pair, r_max, d_srf threshold) in that nesting order a record
 *   rdf[n_bins] | knn[k_max][n_bins] | meta[PS_META_LEN(k_max)], identical to
 *   ps_spatstat with the same parameters (entries past that r_max's bins are 0).
 *   No host synchronisation: the sequence can be captured in a CUDA graph.
 */
typedef struct {
  const float* xyz;
  const uint8_t* type;
  const float* dsrf;
  int64_t n;
} ps_dataset;

typedef struct {
  uint32_t struct_size;
  ps_bins bins;
  uint32_t n_rmax;
  uint32_t rmax_bins[4];
  uint32_t n_dsrf;
  float dsrf_min[4];
  uint32_t n_pairs;
  uint64_t ctr_mask[4][4];
  uint64_t nbr_mask[4][4];
  uint32_t k_max;
  float cell_scale;
} ps_sweep;

typedef struct ps_batch ps_batch;
PS_API int ps_batch_create(const ps_dataset* datasets, int n_datasets, const ps_sweep* sweep, ps_batch** out);
PS_API int ps_batch_run(ps_batch* b, uint64_t* d_out, void* stream);
PS_API int64_t ps_batch_out_len(const ps_batch* b);
PS_API int ps_batch_destroy(ps_batch* b);

/*
 * Gaussian-smoothed RDF and its adjoint (the differentiable form).  The paper
 * bins with rectangular transfer functions (Methods, "Descriptive, two-point
 * spatial statistics, and clustering"); here each pair's distance is smoothed
 * by a Gaussian of width sigma and integrated over every bin:
 *   u_ij = scale * |x_j - x_i|   (float32 coordinates; pairs j != i, j in the
 *                                  grid's neighbour set, i central as above)
 *   h[b] = sum over pairs with u_ij < stop + 6 sigma of
 *          Phi((e_{b+1} - u_ij)/sigma) - Phi((e_b - u_ij)/sigma),  e_b = r0 + b*dr
 * ps_rdf_soft_fwd writes float32 h[n_bins] (d_h, device).
 * ps_rdf_soft_bwd takes d_dLdh = dL/dh (float32 [n_bins], device) and writes
 *   d_grad_xyz  float32 [n][3]: dL/dx for every ion of the grid's cloud
 *               (zero for ions in no pair), overwritten
 *   d_grad_scale float32 [1]: dL/dscale
 * Pairs are recomputed in the adjoint, never stored.  The grid must have been
 * built with r_cut * scale >= stop + 6 sigma (PS_ERR_INVALID_ARG otherwise) and
 * must be rebuilt when the positions change.  The central set is chosen by
 * d_srf at scale 1 and does not depend on scale.  Accuracy: float32 arithmetic
 * on a fine grid of width <= sigma/40 with a second-order expansion per pair
 * (relative error ~1e-6 of h and of the gradient).  Device-side input errors
 * are reported by ps_grid_get_info.
 */
PS_API int ps_rdf_soft_fwd(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma,
                           float scale, ps_bins bins, float* d_h, void* stream);
PS_API int ps_rdf_soft_bwd(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma,
                           float scale, ps_bins bins, const float* d_dLdh, float* d_grad_xyz, float* d_grad_scale,
                           void* stream);

/*
 * Spatial distribution map: the three-dimensional two-point statistic (Methods,
 * "Descriptive, two-point spatial statistics, and clustering": RDF and kNN are
 * its annular integrals; Results on strong scaling: cubic voxels of
 * (0.025 nm)^3 about every central ion, ROI radius R = 2 nm).
 *   For every central i (type in ctr_mask, d_srf >= dsrf_min) and neighbour
 *   j != i of the grid's set with d2_ij < (float)(r_max^2), the float32
 *   displacement (dx, dy, dz) = x_j - x_i lands in voxel (mx, my, mz) with
 *   V[m] <= d < V[m+1] on each axis, V[m] = (float)((m - n_vox/2) * w)
 *   computed in double, m = 0..n_vox.
 *   g        grid built with r_cut >= r_max (else PS_ERR_INVALID_ARG)
 *   spec     r_max > 0, w > 0, 1 <= n_vox <= PS_SDM_MAX_VOX
 *   d_hist   device uint64 [n_vox][n_vox][n_vox], index (mz*n_vox + my)*n_vox + mx
 *   d_meta   device uint64 [PS_SDM_META_LEN]: n_central, pairs in the map,
 *            pairs whose displacement lies outside the voxel cube, status
 * Both outputs are overwritten.  Asynchronous on `stream`.
 */
#define PS_SDM_MAX_VOX 1024
#define PS_SDM_META_LEN 4
typedef struct {
  double r_max; /* ROI radius (nm) */
  double w;     /* voxel edge (nm) */
  uint32_t n_vox;
} ps_sdm_spec;
PS_API int ps_sdm(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_sdm_spec spec,
                  uint64_t* d_hist, uint64_t* d_meta, void* stream);

/*
 * Maximum-separation clustering (Methods, "Descriptive, two-point spatial
 * statistics, and clustering": the DBScan variant with threshold distance
 * d_max and minimum cluster size N_min; Results on the AM specimens for the
 * d_max sweeps and the clusters truncated by the dataset edge).
 *   The ions of the grid's set (its neighbour types) are linked when
 *   d2 <= (float)(d_max^2) (float32 d2 as in ps_spatstat); clusters are the
 *   connected components with at least n_min ions.
 *   g        grid built with r_cut >= d_max (else PS_ERR_INVALID_ARG); its
 *            central-list storage is used as scratch (later queries rebuild it)
 *   dsrf     device float32 [n] or NULL: a cluster is "interior" when all its
 *            ions have d_srf >= spec.dsrf_min (NULL: every cluster)
 *   d_label  device uint32 [n]: the smallest original index of the ion's
 *            cluster, or 0xFFFFFFFF (other types, or a component below n_min)
 *   d_size_hist, d_interior_hist  device uint64 [hist_len]: clusters by size
 *            (sizes >= hist_len - 1 in the last entry), all / interior only
 *   d_meta   device uint64 [PS_CLUSTER_META_LEN]: ions in the set, clusters,
 *            ions in clusters, interior clusters, status
 * All outputs are overwritten.  Asynchronous on `stream`.  n < 2^32 - 1.
 */
#define PS_CLUSTER_META_LEN 5
typedef struct {
  double d_max;     /* link distance (nm) */
  uint32_t n_min;   /* smallest cluster, >= 1 */
  float dsrf_min;   /* interior threshold on d_srf */
  uint32_t hist_len; /* >= 2 */
} ps_cluster_spec;
PS_API int ps_cluster(ps_grid* g, const float* dsrf, ps_cluster_spec spec, uint32_t* d_label, uint64_t* d_size_hist,
                      uint64_t* d_interior_hist, uint64_t* d_meta, void* stream);

/*
 * Randomised type labels: the paper computes every statistic also for a
 * random relabelling of the ions, as the reference for a random arrangement
 * (Suppl. "Importance of high quality random number generators").
 *   type_out[i] = type_in[perm(i)], perm a pseudo-random permutation of
 *   [0, n) fixed by seed: a 4-round Feistel network on 2h bits (2^(2h) >= n,
 *   h >= 1), round function = splitmix64 finaliser of (half-block + key_r),
 *   key_r = finaliser(seed + (r + 1) * 0x9e3779b97f4a7c15), restricted to
 *   [0, n) by cycle walking.  Label counts are kept exactly.
 * type_in, type_out: device uint8 [n] (distinct); d_perm: optional device
 * uint32 [n] receiving perm.  Run the statistics on type_out for the
 * randomised companion.  n < 2^32.
 */
PS_API int ps_shuffle_labels(const uint8_t* type_in, uint8_t* type_out, int64_t n, uint64_t seed, uint32_t* d_perm,
                             void* stream);

/*
 * Allocation-free ps_build_grid + ps_spatstat.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory while
 * they run the statistics, e.g. applications that give all device memory to
 * their own pool at start-up (a cudaMalloc inside the library would fail) or
 * acquisition loops that cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree.
 *   - Scratch is one file-scope device array sized for PS_STATIC_MAX_IONS
 *     ions (about 14 MB), held on every GPU that uses the library until the
 *     process exits.  No cudaMalloc, cudaFree or other allocating routine is
 *     called.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *   - n > PS_STATIC_MAX_IONS returns PS_ERR_CAPACITY, n < 0 PS_ERR_INVALID_ARG;
 *     every argument check of ps_grid_build and ps_spatstat is made before any
 *     work is enqueued, so a refused call leaves the scratch untouched.
 *   - Every call on a device shares the one array, which keeps the last call's
 *     contents (each call clears what must start at zero).  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race and give
 *     wrong results: serialise them.
 *   - Cells of edge >= r_cut (the 27-cell search); arguments and outputs as
 *     in ps_grid_build and ps_spatstat.
 */
#define PS_STATIC_MAX_IONS 262144
PS_API int ps_spatstat_static(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n,
                              const uint64_t nbr_mask[4], float r_cut, const uint64_t ctr_mask[4], float dsrf_min,
                              ps_bins bins, const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn,
                              uint64_t* d_meta, float* d_kth, uint32_t* d_nwithin, void* stream);

/*
 * Launch accounting and per-kernel timing (no counterpart in the paper; the
 * paper reports wall-clock per task).
 *   ps_launch_count   kernels this library has launched in this process.
 *   ps_prof_enable    record a CUDA event pair on the launching stream around
 *                     every launch of the kernel families in `kid_mask`
 *                     (bit 1 << PS_KID_*); 0 disables.  Resets the tallies.
 *                     Synchronises the device.
 *   ps_prof_read      launches and summed event time (ms) of one family since
 *                     ps_prof_enable; waits for the recorded events.
 */
typedef enum {
  PS_KID_RESET = 1,      /* grid reset */
  PS_KID_SELECT = 2,     /* neighbour-set selection + bounding box */
  PS_KID_GEOMETRY = 3,   /* cell geometry + zeroing of the counts */
  PS_KID_COUNT = 4,      /* cell index + rank of the neighbours */
  PS_KID_SCAN = 5,       /* exclusive scans of cell counts and the central lists' cell starts */
  PS_KID_SCATTER = 6,    /* counting-sort scatters (neighbours; vertex-centred centrals) */
  PS_KID_CENTRAL = 7,    /* central reset + selection + cell rank (and the vertex-centred count) */
  PS_KID_QUERY = 8,      /* exact kNN + RDF query (the split query's near-radius kNN pass) */
  PS_KID_EPILOGUE = 9,   /* meta epilogue */
  PS_KID_SOFT_FWD = 10,  /* smoothed RDF forward */
  PS_KID_SOFT_BWD = 11,  /* smoothed RDF adjoint */
  PS_KID_BATCH = 12,     /* batched sweep kernels */
  PS_KID_LABELS = 13,    /* randomised labels */
  PS_KID_SDM = 14,       /* spatial distribution map */
  PS_KID_CLUSTER = 15,   /* maximum-separation clustering */
  PS_KID_FINALISE = 16,  /* g(r) normalisation */
  PS_KID_PEAKS = 17,     /* throughput microbenchmarks (ps_measure_peaks) */
  PS_KID_RDF_SYM = 18,   /* RDF over unordered pairs (the split query's third pass) */
  PS_KID_KNN_FULL = 19,  /* full-radius kNN of the centrals the near pass left (split query) */
  PS_KID_COUNT_ = 20
} ps_kernel_id;
PS_API uint64_t ps_launch_count(void);

/*
 * Measured throughput of the units the statistics are bound by (no
 * counterpart in the paper): the denominators of the query's rooflines on the
 * GPU at hand.  Runs three short microbenchmarks on `stream` (a few ms each,
 * best of three) and synchronises; allocates and frees a few KB.
 *   fp32_scalar_gops  1e9 float32 add/multiply results per second with scalar
 *                     instructions (no fused multiply-add: the pair test is
 *                     ((dx*dx)+(dy*dy))+(dz*dz), never contracted)
 *   fp32_packed_gops  the same with packed f32x2 instructions
 *   smem_atomic_gops  1e9 32-bit shared-memory atomic adds per second, every
 *                     lane on its own bank (the conflict-free rate)
 *   sm_mhz            SM clock during the runs (clock64 ticks per ns)
 *   num_sms           multiprocessors of the current device
 * out->struct_size must be sizeof(ps_peaks).
 */
typedef struct {
  uint32_t struct_size;
  int32_t num_sms;
  double fp32_scalar_gops;
  double fp32_packed_gops;
  double smem_atomic_gops;
  double sm_mhz;
} ps_peaks;
PS_API int ps_measure_peaks(ps_peaks* out, void* stream);

/*
 * Failure detection hooks for tests (no counterpart in the paper; the library's
 * own convention that every failure returns a status and leaks nothing).
 *   ps_debug_fail_alloc   the nth device allocation of the library from now on
 *                         fails as if the device were out of memory (1 = the
 *                         next one; 0 disarms).  The failing call must return
 *                         PS_ERR_OOM and free whatever it had allocated.
 *   ps_debug_live_allocs  device allocations of the library not yet freed.
 *   ps_debug_wait_selftest  runs the library's two bounded device waits -- the
 *                         look-back of the single-pass scans and the mbarrier
 *                         wait of the bulk copies -- on events that never
 *                         happen, each giving up after limit_ns (<= 2 s).
 *                         d_work: device uint64 [4], overwritten; afterwards
 *                         d_work[2] (look-back) and d_work[3] (mbarrier) hold
 *                         PS_ERR_TIMEOUT.  Nothing is left in flight.
 */
PS_API int ps_debug_fail_alloc(int64_t nth);
PS_API int64_t ps_debug_live_allocs(void);
PS_API int ps_debug_wait_selftest(uint64_t limit_ns, uint64_t* d_work, void* stream);
PS_API int ps_prof_enable(uint32_t kid_mask);
PS_API int ps_prof_read(uint32_t kid, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* PS_H */
