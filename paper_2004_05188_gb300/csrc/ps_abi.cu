// C ABI entry points of libps: argument checks, handle lifetime, dispatch.
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include "ps_internal.cuh"

namespace ps {

static thread_local std::string t_error;

void set_error(const std::string& msg) { t_error = msg; }

int fail(int code, const std::string& msg) {
  t_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  t_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
}

// Every device allocation of the library goes through dev_malloc / dev_free: they keep the
// count of live allocations and host the failure injection of ps_debug_fail_alloc.
static std::atomic<int64_t> g_fail_countdown{0};
static std::atomic<int64_t> g_live_allocs{0};

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  int64_t c = g_fail_countdown.load();
  while (c > 0 && !g_fail_countdown.compare_exchange_weak(c, c - 1)) {
  }
  if (c == 1) return cudaErrorMemoryAllocation;  // the injected failure: nothing is allocated
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  const cudaError_t e = cudaFree(p);
  if (e == cudaSuccess) g_live_allocs.fetch_sub(1);
  return e;
}

int wait_selftest(uint64_t limit_ns, unsigned long long* d_work, cudaStream_t s);

int run_query(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
              const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn, uint64_t* d_meta, float* d_kth,
              uint32_t* d_nwithin, cudaStream_t s);

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void edges_host(ps_bins b, float* E) {
  for (uint32_t i = 0; i <= b.n_bins; ++i) {
    const double e = b.r0 + (double)i * b.dr;
    E[i] = (float)(e * e);
  }
}

static int check_bins(ps_bins b) {
  if (!(b.dr > 0.0) || !(b.r0 >= 0.0) || !std::isfinite(b.dr) || !std::isfinite(b.r0))
    return fail(PS_ERR_INVALID_ARG, "bins: need r0 >= 0 and dr > 0, finite");
  if (b.n_bins < 1 || b.n_bins > PS_MAX_BINS) return fail(PS_ERR_UNSUPPORTED, "bins: n_bins out of range");
  return PS_OK;
}


// Host-side checks of the statistics arguments (everything ps_spatstat refuses before it
// enqueues work), against the cutoff r_cut of the grid the query will search.
int check_spatstat_args(const char* who, const uint64_t* ctr_mask, float dsrf_min, ps_bins bins, const uint32_t* ks,
                        uint32_t n_k, const uint64_t* d_knn, const uint64_t* d_meta, float r_cut) {
  const std::string w(who);
  if (!ctr_mask || !d_meta) return fail(PS_ERR_INVALID_ARG, w + ": ctr_mask/d_meta is NULL");
  int rc = check_bins(bins);
  if (rc) return rc;
  if (n_k > PS_MAX_KLIST) return fail(PS_ERR_UNSUPPORTED, w + ": too many k values");
  if (n_k > 0 && (!ks || !d_knn)) return fail(PS_ERR_INVALID_ARG, w + ": ks/d_knn is NULL");
  for (uint32_t q = 0; q < n_k; ++q)
    if (ks[q] < 1 || ks[q] > PS_K_MAX) return fail(PS_ERR_UNSUPPORTED, w + ": k must be in [1, 32]");
  if (std::isnan(dsrf_min)) return fail(PS_ERR_INVALID_ARG, w + ": dsrf_min is NaN");
  // the largest edge, by the same formula as every kernel: E[n_bins] = (float)((r0 + n_bins dr)^2)
  const double e = bins.r0 + (double)bins.n_bins * bins.dr;
  const float Emax = (float)(e * e);
  if ((double)Emax > (double)r_cut * (double)r_cut)
    return fail(PS_ERR_INVALID_ARG, w + ": the grid's r_cut is below the histogram stop");
  return PS_OK;
}
}  // namespace ps

using namespace ps;

extern "C" {

int ps_version(void) { return 100; }

const char* ps_last_error(void) { return t_error.c_str(); }

int ps_bin_edges(ps_bins bins, float* E) {
  if (!E) return fail(PS_ERR_INVALID_ARG, "ps_bin_edges: E is NULL");
  int rc = check_bins(bins);
  if (rc) return rc;
  edges_host(bins, E);
  return PS_OK;
}

int ps_grid_create(int64_t n_max, const ps_grid_opts* opts, ps_grid** out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "ps_grid_create: out is NULL");
  *out = nullptr;
  if (n_max < 0 || n_max > (int64_t)UINT32_MAX - 1) return fail(PS_ERR_INVALID_ARG, "ps_grid_create: n_max out of range");
  float cell_scale = 1.0f;
  uint32_t block = 0;
  if (opts) {
    if (opts->struct_size < sizeof(uint32_t) + sizeof(float))
      return fail(PS_ERR_INVALID_ARG, "ps_grid_create: opts->struct_size too small");
    if (opts->cell_scale != 0.0f) cell_scale = opts->cell_scale;
    if (opts->struct_size >= offsetof(ps_grid_opts, block) + sizeof(uint32_t)) block = opts->block;
  }
  if (!(cell_scale >= kMinCellScale) || !std::isfinite(cell_scale))
    return fail(PS_ERR_INVALID_ARG, "cell_scale must be >= 1/3");
  ps_grid* g = new (std::nothrow) ps_grid();
  if (!g) return fail(PS_ERR_OOM, "host allocation failed");
  g->n_max = n_max > 0 ? n_max : 1;
  g->cell_scale = cell_scale;
  g->stencil = cell_scale >= 1.0f ? 1 : (cell_scale >= 0.5f ? 2 : 3);
  g->block = block;
  if (opts && opts->struct_size >= offsetof(ps_grid_opts, dense_min) + sizeof(uint32_t))
    g->dense_min = opts->dense_min ? opts->dense_min : 0xFFFFFFFFu;
  if (opts && opts->struct_size >= offsetof(ps_grid_opts, split) + sizeof(uint32_t)) g->split = opts->split != 0;
  // cells: a bounding-box grid at the cutoff needs ~n/100 cells for the clouds seen here; the
  // capacity leaves a wide margin (the cell edge grows past it, results do not change)
  const int64_t cap0 = g->stencil >= 2 ? g->n_max : g->n_max / 8;
  const int64_t cap = cap0 > 65536 ? cap0 : 65536;
  g->cell_cap = (uint32_t)(cap < (int64_t)1 << 31 ? cap : (int64_t)1 << 31);
  // scan tiles of 4096 cells or 4096 records (the central list's record compaction)
  g->scan_tiles_cap = (uint32_t)(((int64_t)g->cell_cap > g->n_max + 1 ? (int64_t)g->cell_cap : g->n_max + 1) + 4095) / 4096;
  const size_t nm = (size_t)g->n_max, cc = g->cell_cap;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t o_sel = take(nm * 4), o_cr = take(nm * 8);
  const size_t o_ncount = take(cc * 4), o_nstart = take((cc + 1) * 4), o_nrec = take(nm * 16);
  const size_t o_ccount = take(cc * 4), o_cstart = take((cc + 1) * 4), o_crec = take(nm * 16), o_cwork = take(cc * 4);
  g->item_cap = (uint32_t)(cc + nm / 8 + 2);  // batches of >= 8 centrals (4 lanes per central) + one per cell
  const size_t o_witem = take((size_t)g->item_cap * 8), o_nwitem = take((size_t)g->item_cap * 8);
  const size_t o_sm0 = take(kSoftFineMax * 8), o_sm1 = take(kSoftFineMax * 8), o_sm2 = take(kSoftFineMax * 8);
  const size_t o_sT = take(3 * kSoftFineMax * 4), o_sgs = take(8);
  const size_t o_part = take((size_t)g->scan_tiles_cap * 8), o_sctr = take(8);
  const size_t o_ngeo = take(sizeof(Geo)), o_cgeo = take(sizeof(Geo));
  void* base = nullptr;
  cudaError_t e = dev_malloc(&base, off);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "cudaMalloc(grid scratch)");
  }
  e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e != cudaSuccess) {
    dev_free(base);
    delete g;
    return cuda_fail(e, "cudaGetDevice");
  }
  char* b = static_cast<char*>(base);
  g->dev_block = base;
  g->sel = reinterpret_cast<uint32_t*>(b + o_sel);
  g->cr = reinterpret_cast<uint2*>(b + o_cr);
  g->nbr.count = reinterpret_cast<uint32_t*>(b + o_ncount);
  g->nbr.start = reinterpret_cast<uint32_t*>(b + o_nstart);
  g->nbr.rec = reinterpret_cast<float4*>(b + o_nrec);
  g->nbr.geo = reinterpret_cast<Geo*>(b + o_ngeo);
  g->ctr.count = reinterpret_cast<uint32_t*>(b + o_ccount);
  g->ctr.start = reinterpret_cast<uint32_t*>(b + o_cstart);
  g->ctr.rec = reinterpret_cast<float4*>(b + o_crec);
  g->ctr.work = reinterpret_cast<uint32_t*>(b + o_cwork);
  g->ctr.witem = reinterpret_cast<uint2*>(b + o_witem);
  g->nbr_witem = reinterpret_cast<uint2*>(b + o_nwitem);
  g->soft_m0 = reinterpret_cast<unsigned long long*>(b + o_sm0);
  g->soft_m1 = reinterpret_cast<double*>(b + o_sm1);
  g->soft_m2 = reinterpret_cast<double*>(b + o_sm2);
  g->soft_T = reinterpret_cast<float*>(b + o_sT);
  g->soft_gs = reinterpret_cast<double*>(b + o_sgs);
  g->ctr.geo = reinterpret_cast<Geo*>(b + o_cgeo);
  g->scan_state = reinterpret_cast<unsigned long long*>(b + o_part);
  g->scan_ctr = reinterpret_cast<uint32_t*>(b + o_sctr);
  e = cudaMemset(g->nbr.geo, 0, sizeof(Geo));
  if (e == cudaSuccess) e = cudaMemset(g->scan_state, 0, (size_t)g->scan_tiles_cap * 8);
  if (e == cudaSuccess) e = cudaMemset(g->scan_ctr, 0, 8);
  if (e == cudaSuccess) e = cudaMemset(g->ctr.geo, 0, sizeof(Geo));
  if (e != cudaSuccess) {
    dev_free(base);
    delete g;
    return cuda_fail(e, "cudaMemset(grid)");
  }
  *out = g;
  return PS_OK;
}

int ps_grid_set_query_opts(ps_grid* g, uint32_t dense_min, uint32_t split) {
  if (!g) return fail(PS_ERR_INVALID_ARG, "ps_grid_set_query_opts: grid is NULL");
  g->dense_min = dense_min ? dense_min : 0xFFFFFFFFu;
  g->split = split != 0;
  return PS_OK;
}

int ps_grid_destroy(ps_grid* g) {
  if (!g) return PS_OK;
  cudaError_t e = cudaSuccess;
  if (g->dev_block) {
    e = cudaDeviceSynchronize();
    cudaError_t e2 = dev_free(g->dev_block);
    if (e == cudaSuccess) e = e2;
  }
  delete g;
  if (e != cudaSuccess) return cuda_fail(e, "ps_grid_destroy");
  return PS_OK;
}

int ps_grid_build(ps_grid* g, const float* xyz, const uint8_t* type, int64_t n, const uint64_t nbr_mask[4],
                  float r_cut, void* stream) {
  if (!g) return fail(PS_ERR_INVALID_ARG, "ps_grid_build: grid is NULL");
  if (n < 0) return fail(PS_ERR_INVALID_ARG, "ps_grid_build: n < 0");
  if (n > g->n_max) return fail(PS_ERR_CAPACITY, "ps_grid_build: n exceeds the grid capacity");
  if (n > 0 && (!xyz || !type)) return fail(PS_ERR_INVALID_ARG, "ps_grid_build: xyz/type is NULL");
  if (!nbr_mask) return fail(PS_ERR_INVALID_ARG, "ps_grid_build: nbr_mask is NULL");
  if (!(r_cut > 0.0f) || !std::isfinite(r_cut)) return fail(PS_ERR_INVALID_ARG, "ps_grid_build: r_cut must be > 0");
  g->xyz = xyz;
  g->type = type;
  g->n = n;
  g->r_cut = r_cut;
  g->built = false;
  int rc = build_neighbour_grid(g, nbr_mask, r_cut, static_cast<cudaStream_t>(stream));
  if (rc == PS_OK) g->built = true;
  return rc;
}

int ps_build_grid(const float* xyz, const uint8_t* type, int64_t n, const uint64_t nbr_mask[4], float r_cut,
                  const ps_grid_opts* opts, void* stream, ps_grid** out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "ps_build_grid: out is NULL");
  int rc = ps_grid_create(n, opts, out);
  if (rc) return rc;
  rc = ps_grid_build(*out, xyz, type, n, nbr_mask, r_cut, stream);
  if (rc) {
    ps_grid_destroy(*out);
    *out = nullptr;
  }
  return rc;
}

int ps_grid_get_info(ps_grid* g, ps_grid_info* info, void* stream) {
  if (!g || !info) return fail(PS_ERR_INVALID_ARG, "ps_grid_get_info: NULL argument");
  if (info->struct_size < sizeof(ps_grid_info)) return fail(PS_ERR_INVALID_ARG, "ps_grid_get_info: struct_size");
  Geo h, hc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PS_CUDA(cudaMemcpyAsync(&h, g->nbr.geo, sizeof(Geo), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&hc, g->ctr.geo, sizeof(Geo), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  if (h.status == 0) h.status = hc.status;
  for (int a = 0; a < 3; ++a) info->dims[a] = h.dims[a], info->origin[a] = h.origin[a];
  info->cell = h.h;
  info->n_nbr = h.n_sel;
  info->n_cells = h.n_cells;
  info->status = h.status;
  return PS_OK;
}

int ps_spatstat(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
                const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn, uint64_t* d_meta, float* d_kth,
                uint32_t* d_nwithin, void* stream) {
  if (!g || !g->built) return fail(PS_ERR_INVALID_ARG, "ps_spatstat: grid is NULL or not built");
  int rc = check_spatstat_args("ps_spatstat", ctr_mask, dsrf_min, bins, ks, n_k, d_knn, d_meta, g->r_cut);
  if (rc) return rc;
  return run_query(g, dsrf, ctr_mask, dsrf_min, bins, ks, n_k, d_rdf, d_knn, d_meta, d_kth, d_nwithin,
                   static_cast<cudaStream_t>(stream));
}

int ps_sdm(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_sdm_spec spec,
           uint64_t* d_hist, uint64_t* d_meta, void* stream) {
  if (!g || !g->built) return fail(PS_ERR_INVALID_ARG, "ps_sdm: grid is NULL or not built");
  if (!ctr_mask || !d_hist || !d_meta) return fail(PS_ERR_INVALID_ARG, "ps_sdm: ctr_mask/d_hist/d_meta is NULL");
  if (std::isnan(dsrf_min)) return fail(PS_ERR_INVALID_ARG, "ps_sdm: dsrf_min is NaN");
  if (!(spec.r_max > 0.0) || !std::isfinite(spec.r_max) || !(spec.w > 0.0) || !std::isfinite(spec.w))
    return fail(PS_ERR_INVALID_ARG, "ps_sdm: r_max and w must be positive and finite");
  if (spec.n_vox < 1 || spec.n_vox > PS_SDM_MAX_VOX) return fail(PS_ERR_UNSUPPORTED, "ps_sdm: n_vox must be in [1, 1024]");
  const float ER = (float)(spec.r_max * spec.r_max);
  if ((double)ER > (double)g->r_cut * (double)g->r_cut)
    return fail(PS_ERR_INVALID_ARG, "ps_sdm: the grid's r_cut is below r_max");
  return run_sdm(g, dsrf, ctr_mask, dsrf_min, spec, d_hist, d_meta, static_cast<cudaStream_t>(stream));
}

int ps_cluster(ps_grid* g, const float* dsrf, ps_cluster_spec spec, uint32_t* d_label, uint64_t* d_size_hist,
               uint64_t* d_interior_hist, uint64_t* d_meta, void* stream) {
  if (!g || !g->built) return fail(PS_ERR_INVALID_ARG, "ps_cluster: grid is NULL or not built");
  if (!d_label || !d_size_hist || !d_interior_hist || !d_meta)
    return fail(PS_ERR_INVALID_ARG, "ps_cluster: an output pointer is NULL");
  if (!(spec.d_max > 0.0) || !std::isfinite(spec.d_max)) return fail(PS_ERR_INVALID_ARG, "ps_cluster: d_max must be > 0");
  if (spec.n_min < 1 || spec.hist_len < 2) return fail(PS_ERR_INVALID_ARG, "ps_cluster: n_min >= 1 and hist_len >= 2");
  if (std::isnan(spec.dsrf_min)) return fail(PS_ERR_INVALID_ARG, "ps_cluster: dsrf_min is NaN");
  if (g->n >= (int64_t)0xFFFFFFFF) return fail(PS_ERR_UNSUPPORTED, "ps_cluster: n must be below 2^32 - 1");
  const float D = (float)(spec.d_max * spec.d_max);
  if ((double)D > (double)g->r_cut * (double)g->r_cut)
    return fail(PS_ERR_INVALID_ARG, "ps_cluster: the grid's r_cut is below d_max");
  return run_cluster(g, dsrf, spec, d_label, d_size_hist, d_interior_hist, d_meta, static_cast<cudaStream_t>(stream));
}

static int check_soft(ps_grid* g, const uint64_t* ctr_mask, ps_bins bins, float dsrf_min) {
  if (!g || !g->built) return fail(PS_ERR_INVALID_ARG, "smoothed RDF: grid is NULL or not built");
  if (!ctr_mask) return fail(PS_ERR_INVALID_ARG, "smoothed RDF: ctr_mask is NULL");
  if (std::isnan(dsrf_min)) return fail(PS_ERR_INVALID_ARG, "smoothed RDF: dsrf_min is NaN");
  return check_bins(bins);
}

int ps_rdf_soft_fwd(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma,
                    float scale, ps_bins bins, float* d_h, void* stream) {
  int rc = check_soft(g, ctr_mask, bins, dsrf_min);
  if (rc) return rc;
  if (!d_h) return fail(PS_ERR_INVALID_ARG, "ps_rdf_soft_fwd: d_h is NULL");
  return soft_forward(g, dsrf, ctr_mask, dsrf_min, sigma, scale, bins, d_h, static_cast<cudaStream_t>(stream));
}

int ps_rdf_soft_bwd(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma,
                    float scale, ps_bins bins, const float* d_dLdh, float* d_grad_xyz, float* d_grad_scale,
                    void* stream) {
  int rc = check_soft(g, ctr_mask, bins, dsrf_min);
  if (rc) return rc;
  if (!d_dLdh || !d_grad_xyz || !d_grad_scale)
    return fail(PS_ERR_INVALID_ARG, "ps_rdf_soft_bwd: d_dLdh/d_grad_xyz/d_grad_scale is NULL");
  return soft_backward(g, dsrf, ctr_mask, dsrf_min, sigma, scale, bins, d_dLdh, d_grad_xyz, d_grad_scale,
                       static_cast<cudaStream_t>(stream));
}

int ps_rdf_normalise(ps_grid* g, const uint64_t* d_meta, const uint64_t* d_rdf, double volume, ps_bins bins,
                     double* d_g, double* d_factor, void* stream) {
  if (!g || !g->built) return fail(PS_ERR_INVALID_ARG, "ps_rdf_normalise: grid is NULL or not built");
  if (!d_meta) return fail(PS_ERR_INVALID_ARG, "ps_rdf_normalise: d_meta is NULL");
  if (!d_g && !d_factor) return fail(PS_ERR_INVALID_ARG, "ps_rdf_normalise: d_g and d_factor are both NULL");
  if (d_g && !d_rdf) return fail(PS_ERR_INVALID_ARG, "ps_rdf_normalise: d_g needs d_rdf");
  if (!(volume > 0.0) || !std::isfinite(volume)) return fail(PS_ERR_INVALID_ARG, "ps_rdf_normalise: volume must be > 0");
  int rc = check_bins(bins);
  if (rc) return rc;
  return rdf_normalise(g, d_meta, d_rdf, volume, bins, d_g, d_factor, static_cast<cudaStream_t>(stream));
}

int ps_knn_hist(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, uint32_t k, ps_bins bins,
                uint64_t* d_hist, uint64_t* d_meta, float* d_kth, void* stream) {
  if (!d_hist) return fail(PS_ERR_INVALID_ARG, "ps_knn_hist: d_hist is NULL");
  return ps_spatstat(g, dsrf, ctr_mask, dsrf_min, bins, &k, 1, nullptr, d_hist, d_meta, d_kth, nullptr, stream);
}

int ps_rdf_hist(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
                uint64_t* d_hist, uint64_t* d_meta, void* stream) {
  if (!d_hist) return fail(PS_ERR_INVALID_ARG, "ps_rdf_hist: d_hist is NULL");
  return ps_spatstat(g, dsrf, ctr_mask, dsrf_min, bins, nullptr, 0, d_hist, nullptr, d_meta, nullptr, nullptr,
                     stream);
}

int ps_debug_fail_alloc(int64_t nth) {
  if (nth < 0) return fail(PS_ERR_INVALID_ARG, "ps_debug_fail_alloc: nth < 0");
  g_fail_countdown.store(nth);
  return PS_OK;
}

int64_t ps_debug_live_allocs(void) { return g_live_allocs.load(); }

int ps_debug_wait_selftest(uint64_t limit_ns, uint64_t* d_work, void* stream) {
  if (!d_work) return fail(PS_ERR_INVALID_ARG, "ps_debug_wait_selftest: d_work is NULL");
  if (limit_ns > kWaitLimitNs) return fail(PS_ERR_INVALID_ARG, "ps_debug_wait_selftest: limit_ns above 2 s");
  return wait_selftest(limit_ns, reinterpret_cast<unsigned long long*>(d_work), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
