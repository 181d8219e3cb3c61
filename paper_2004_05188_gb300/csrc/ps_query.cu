// Exact kNN + RDF query over the cell grid.
//
// The paper evaluates one spherical ROI per central ion and machines the ROIs
// off with a dynamic schedule, each thread keeping its own result buffers that
// are merged afterwards (Suppl. "Customized user defined batch processing
// queues").  Here a persistent CTA takes one non-empty central cell at a time
// from a device work counter (the dynamic schedule), stages the 27 neighbour
// cells of that cell into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier), and evaluates every central of
// the cell against the staged records.  Results go to per-CTA shared-memory
// histograms (the per-thread buffers) that are added to the uint64 global
// histograms once per CTA.
//
// Two mappings of centrals to threads, chosen per cell:
//   A (dense cells):  one thread per central, the whole block walks the
//                     staged candidates in lock step (shared-memory broadcast);
//   B (sparse cells): one warp per central, lanes stride over the candidates,
//                     per-lane top-k lists merged by warp shuffles.
// Both keep the k smallest squared distances in registers (sorted insertion).
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

struct QueryArgs {
  const float4* nrec;
  const uint32_t* nstart;
  const Geo* ngeo;
  const float4* crec;
  const uint32_t* cstart;
  const uint32_t* cwork;
  Geo* cgeo;
  double r0, dr;
  uint32_t n_bins;
  uint32_t n_k;
  uint32_t k_need;  // max requested k
  uint32_t stage_cap;  // float4 records per staging chunk
  uint32_t ks[PS_MAX_KLIST];
  uint64_t* rdf;
  uint64_t* knn;
  uint64_t* meta;
  float* kth;
  uint32_t* nwithin;
  int64_t n;  // ions in the cloud (stride of kth)
};

constexpr uint32_t kModeAMin = 64;  // cells with at least this many centrals use mapping A

template <int K>
__device__ __forceinline__ void topk_insert(float (&top)[K], float x) {
  if (x < top[K - 1]) {
#pragma unroll
    for (int t = K - 1; t > 0; --t) top[t] = fminf(top[t], fmaxf(x, top[t - 1]));
    top[0] = fminf(top[0], x);
  }
}

template <int K>
__device__ __forceinline__ float topk_get(const float (&top)[K], uint32_t idx) {
  float v = INFINITY;
#pragma unroll
  for (int t = 0; t < K; ++t)
    if ((uint32_t)t == idx) v = top[t];
  return v;
}

// bin b in [0, nb) with sE[b] <= d2 < sE[b+1]; caller guarantees sE[0] <= d2 < sE[nb]
__device__ __forceinline__ uint32_t bin_index(float d2, const float* sE, uint32_t nb, float r0f, float inv_dr) {
  const float g = (__fsqrt_rn(d2) - r0f) * inv_dr;
  int b = (int)g;
  b = b < 0 ? 0 : (b >= (int)nb ? (int)nb - 1 : b);
  while (b > 0 && d2 < sE[b]) --b;
  while (b + 1 < (int)nb && d2 >= sE[b + 1]) ++b;
  return (uint32_t)b;
}

struct SmemLayout {
  uint32_t off_E, off_rdf, off_knn, off_kmeta, off_stage, total;
};

__host__ __device__ inline SmemLayout smem_layout(uint32_t n_bins, uint32_t n_k, bool rdf, uint32_t stage_cap) {
  SmemLayout L;
  uint32_t o = 0;
  L.off_E = o;
  o += (n_bins + 1) * 4;
  L.off_rdf = o;
  o += rdf ? n_bins * 4 : 0;
  L.off_knn = o;
  o += n_k * n_bins * 4;
  L.off_kmeta = o;
  o += n_k * 2 * 4;
  o = (o + 15u) & ~15u;
  L.off_stage = o;
  o += stage_cap * 16;
  L.total = o;
  return L;
}

template <int KMAX, bool RDF>
__global__ void __launch_bounds__(256) k_query(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t s_item;
  __shared__ uint32_t s_run_src[9], s_run_len[9];
  __shared__ int s_timeout;

  const SmemLayout L = smem_layout(a.n_bins, a.n_k, RDF, a.stage_cap);
  float* sE = reinterpret_cast<float*>(smem + L.off_E);
  uint32_t* s_rdf = reinterpret_cast<uint32_t*>(smem + L.off_rdf);
  uint32_t* s_knn = reinterpret_cast<uint32_t*>(smem + L.off_knn);
  uint32_t* s_kmeta = reinterpret_cast<uint32_t*>(smem + L.off_kmeta);
  float4* s_cand = reinterpret_cast<float4*>(smem + L.off_stage);

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const uint32_t nb = a.n_bins;
  // edge table: the same double formula as the host, E[b] = (float)((r0 + b*dr)^2)
  for (uint32_t b = tid; b <= nb; b += blockDim.x) {
    const double e = __dadd_rn(a.r0, __dmul_rn((double)b, a.dr));
    sE[b] = __double2float_rn(__dmul_rn(e, e));
  }
  if (RDF)
    for (uint32_t b = tid; b < nb; b += blockDim.x) s_rdf[b] = 0;
  for (uint32_t b = tid; b < a.n_k * nb; b += blockDim.x) s_knn[b] = 0;
  for (uint32_t b = tid; b < 2 * a.n_k; b += blockDim.x) s_kmeta[b] = 0;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_timeout = 0;
  }
  __syncthreads();

  const float Emax = sE[nb], E0 = sE[0];
  const float r0f = (float)a.r0, inv_dr = (float)(1.0 / a.dr);
  const Geo ng = *a.ngeo;
  const uint32_t work_n = a.cgeo->work_n;
  uint32_t phase = 0;
  uint64_t my_binned = 0, my_below = 0;
  uint64_t bound = 0;  // upper bound of any shared counter since the last flush (uniform)

  auto flush = [&]() {
    __syncthreads();
    if (RDF)
      for (uint32_t b = tid; b < nb; b += blockDim.x)
        if (s_rdf[b]) atomicAdd((unsigned long long*)&a.rdf[b], (unsigned long long)s_rdf[b]), s_rdf[b] = 0;
    for (uint32_t b = tid; b < a.n_k * nb; b += blockDim.x)
      if (s_knn[b]) atomicAdd((unsigned long long*)&a.knn[b], (unsigned long long)s_knn[b]), s_knn[b] = 0;
    for (uint32_t b = tid; b < 2 * a.n_k; b += blockDim.x)
      if (s_kmeta[b])
        atomicAdd((unsigned long long*)&a.meta[PS_META_HEAD + b], (unsigned long long)s_kmeta[b]), s_kmeta[b] = 0;
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.cgeo->work_next, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= work_n || s_timeout) break;
    const uint32_t c = a.cwork[item];
    const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
    const uint32_t c0 = a.cstart[c], n_c = a.cstart[c + 1] - c0;
    if (tid < 9) {
      const int y = (int)cy + (int)(tid % 3) - 1, z = (int)cz + (int)(tid / 3) - 1;
      uint32_t src = 0, len = 0;
      if (y >= 0 && z >= 0 && y < (int)ng.dims[1] && z < (int)ng.dims[2]) {
        const uint32_t xlo = cx > 0 ? cx - 1 : 0, xhi = cx + 1 < ng.dims[0] ? cx + 1 : ng.dims[0] - 1;
        const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
        src = a.nstart[row + xlo];
        len = a.nstart[row + xhi + 1] - src;
      }
      s_run_src[tid] = src;
      s_run_len[tid] = len;
    }
    __syncthreads();
    uint32_t n_cand = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r) n_cand += s_run_len[r];

    // bound the shared 32-bit counters: flush before they could overflow
    const uint64_t inc = (uint64_t)n_c * ((uint64_t)n_cand + 1);
    if (bound + inc >= (1ull << 31)) {
      flush();
      bound = 0;
    }
    bound += inc;

    const bool modeA = n_c >= kModeAMin;
    const uint32_t batch = modeA ? blockDim.x : nwarps;
    for (uint32_t cb = 0; cb < n_c; cb += batch) {
      const uint32_t ci = cb + (modeA ? tid : warp);
      const bool valid = ci < n_c;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) p = a.crec[c0 + ci];
      const uint32_t pidx = __float_as_uint(p.w);
      float top[KMAX > 0 ? KMAX : 1];
#pragma unroll
      for (int t = 0; t < (KMAX > 0 ? KMAX : 1); ++t) top[t] = INFINITY;
      uint32_t within = 0;

      // walk the 9 runs in chunks of at most stage_cap records
      uint32_t r = 0, ro = 0;
      while (r < 9) {
        // assemble the next chunk (every thread computes the same pieces)
        uint32_t chunk = 0;
        uint32_t rr = r, rro = ro;
        while (rr < 9 && chunk < a.stage_cap) {
          const uint32_t len = s_run_len[rr];
          const uint32_t take = min(len - rro, a.stage_cap - chunk);
          chunk += take;
          rro += take;
          if (rro >= len) ++rr, rro = 0;
        }
        if (chunk == 0) break;
        if (tid == 0) {
          mbar_arrive_expect_tx(&bar, chunk * 16u);
          uint32_t dst = 0, q = r, qo = ro;
          while (q < 9 && dst < chunk) {
            const uint32_t len = s_run_len[q];
            const uint32_t take = min(len - qo, chunk - dst);
            if (take) bulk_g2s(s_cand + dst, a.nrec + s_run_src[q] + qo, take * 16u, &bar);
            dst += take;
            qo += take;
            if (qo >= len) ++q, qo = 0;
          }
        }
        r = rr;
        ro = rro;
        if (!mbar_wait_bounded(&bar, phase, kWaitLimitNs)) s_timeout = 1;
        phase ^= 1u;

        if (valid) {
          if (modeA) {
            for (uint32_t t = 0; t < chunk; ++t) {
              const float4 q = s_cand[t];
              const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
              if (d2 < Emax && __float_as_uint(q.w) != pidx) {
                ++within;
                if (RDF) {
                  if (d2 >= E0) {
                    atomicAdd(&s_rdf[bin_index(d2, sE, nb, r0f, inv_dr)], 1u);
                    ++my_binned;
                  } else {
                    ++my_below;
                  }
                }
                if (KMAX > 0) topk_insert(top, d2);
              }
            }
          } else {
            for (uint32_t t = lane; t < chunk; t += 32) {
              const float4 q = s_cand[t];
              const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
              if (d2 < Emax && __float_as_uint(q.w) != pidx) {
                ++within;
                if (RDF) {
                  if (d2 >= E0) {
                    atomicAdd(&s_rdf[bin_index(d2, sE, nb, r0f, inv_dr)], 1u);
                    ++my_binned;
                  } else {
                    ++my_below;
                  }
                }
                if (KMAX > 0) topk_insert(top, d2);
              }
            }
          }
        }
        __syncthreads();  // the chunk buffer is reused next
      }

      // finalize the batch's centrals
      if (modeA) {
        if (valid) {
          if (a.nwithin) a.nwithin[pidx] = within;
          if (KMAX > 0)
            for (uint32_t q = 0; q < a.n_k; ++q) {
              const float D = topk_get(top, a.ks[q] - 1);
              if (a.kth) a.kth[(int64_t)q * a.n + pidx] = D;
              if (!(D < Emax))
                atomicAdd(&s_kmeta[2 * q], 1u);
              else if (D < E0)
                atomicAdd(&s_kmeta[2 * q + 1], 1u);
              else
                atomicAdd(&s_knn[q * nb + bin_index(D, sE, nb, r0f, inv_dr)], 1u);
            }
        }
      } else {
        // warp-level: total count and merge of the per-lane sorted lists
        uint32_t w = within;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (valid && lane == 0 && a.nwithin) a.nwithin[pidx] = w;
        if (KMAX > 0) {
          float Dk[PS_MAX_KLIST > 0 ? 1 : 1];
          (void)Dk;
          for (uint32_t rank = 0; rank < a.k_need; ++rank) {
            float m = top[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            const uint32_t bal = __ballot_sync(0xffffffffu, top[0] == m);
            if (lane == (uint32_t)(__ffs(bal) - 1)) {
#pragma unroll
              for (int t = 0; t < (KMAX > 0 ? KMAX : 1) - 1; ++t) top[t] = top[t + 1];
              top[(KMAX > 0 ? KMAX : 1) - 1] = INFINITY;
            }
            if (valid && lane == 0)
              for (uint32_t q = 0; q < a.n_k; ++q) {
                if (a.ks[q] != rank + 1) continue;
                if (a.kth) a.kth[(int64_t)q * a.n + pidx] = m;
                if (!(m < Emax))
                  atomicAdd(&s_kmeta[2 * q], 1u);
                else if (m < E0)
                  atomicAdd(&s_kmeta[2 * q + 1], 1u);
                else
                  atomicAdd(&s_knn[q * nb + bin_index(m, sE, nb, r0f, inv_dr)], 1u);
              }
          }
        }
      }
    }
    __syncthreads();  // s_item and the run table are rewritten next
  }

  flush();
  // pair counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_binned += __shfl_xor_sync(0xffffffffu, my_binned, o);
    my_below += __shfl_xor_sync(0xffffffffu, my_below, o);
  }
  if (lane == 0) {
    if (my_binned) atomicAdd((unsigned long long*)&a.meta[PS_META_N_PAIRS], (unsigned long long)my_binned);
    if (my_below) atomicAdd((unsigned long long*)&a.meta[PS_META_N_BELOW], (unsigned long long)my_below);
  }
  if (tid == 0 && s_timeout) atomicCAS((int*)&a.cgeo->status, 0, (int)PS_ERR_TIMEOUT);
}

// Writes n_central and the device status into the meta array.
__global__ void k_query_epilogue(const Geo* __restrict__ ngeo, const Geo* __restrict__ cgeo, uint64_t* meta) {
  if (threadIdx.x == 0) {
    meta[PS_META_N_CENTRAL] = cgeo->n_sel;
    int st = cgeo->status;
    if (st == 0) st = ngeo->status;
    meta[PS_META_STATUS] = (uint64_t)(uint32_t)st;
  }
}

template <int KMAX, bool RDF>
static int launch_query(const ps_grid* g, const QueryArgs& qa, uint32_t smem, cudaStream_t s) {
  auto kern = k_query<KMAX, RDF>;
  PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
  if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "query kernel does not fit on an SM");
  kern<<<g->num_sms * per_sm, 256, smem, s>>>(qa);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

template <bool RDF>
static int dispatch_k(const ps_grid* g, const QueryArgs& qa, uint32_t smem, cudaStream_t s) {
  const uint32_t k = qa.k_need;
  if (k == 0) return RDF ? launch_query<0, RDF>(g, qa, smem, s) : PS_OK;
  if (k <= 1) return launch_query<1, RDF>(g, qa, smem, s);
  if (k <= 2) return launch_query<2, RDF>(g, qa, smem, s);
  if (k <= 4) return launch_query<4, RDF>(g, qa, smem, s);
  if (k <= 8) return launch_query<8, RDF>(g, qa, smem, s);
  if (k <= 16) return launch_query<16, RDF>(g, qa, smem, s);
  return launch_query<32, RDF>(g, qa, smem, s);
}

int run_query(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
              const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn, uint64_t* d_meta, float* d_kth,
              uint32_t* d_nwithin, cudaStream_t s) {
  QueryArgs qa;
  memset(&qa, 0, sizeof(qa));
  qa.nrec = g->nbr.rec;
  qa.nstart = g->nbr.start;
  qa.ngeo = g->nbr.geo;
  qa.crec = g->ctr.rec;
  qa.cstart = g->ctr.start;
  qa.cwork = g->ctr.work;
  qa.cgeo = g->ctr.geo;
  qa.r0 = bins.r0;
  qa.dr = bins.dr;
  qa.n_bins = bins.n_bins;
  qa.n_k = n_k;
  qa.k_need = 0;
  for (uint32_t q = 0; q < n_k; ++q) {
    qa.ks[q] = ks[q];
    if (ks[q] > qa.k_need) qa.k_need = ks[q];
  }
  qa.rdf = d_rdf;
  qa.knn = d_knn;
  qa.meta = d_meta;
  qa.kth = d_kth;
  qa.nwithin = d_nwithin;
  qa.n = g->n;

  const bool rdf = d_rdf != nullptr;
  PS_CUDA(cudaMemsetAsync(d_meta, 0, PS_META_LEN(n_k) * sizeof(uint64_t), s));
  if (rdf) PS_CUDA(cudaMemsetAsync(d_rdf, 0, (size_t)bins.n_bins * sizeof(uint64_t), s));
  if (n_k) PS_CUDA(cudaMemsetAsync(d_knn, 0, (size_t)n_k * bins.n_bins * sizeof(uint64_t), s));

  int rc = build_central_list(g, dsrf, ctr_mask, dsrf_min, s);
  if (rc) return rc;

  // staging budget: two CTAs per SM
  int dev_smem = 0;
  PS_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  const SmemLayout base = smem_layout(bins.n_bins, n_k, rdf, 0);
  const uint32_t budget = (uint32_t)dev_smem / 2 - 2048;
  if (base.total + 16 * 1024 > (uint32_t)dev_smem - 1024)
    return fail(PS_ERR_UNSUPPORTED, "too many bins x k values for shared memory");
  uint32_t stage_bytes = budget > base.total + 16 * 1024 ? budget - base.total : 16 * 1024;
  qa.stage_cap = stage_bytes / 16;
  const uint32_t smem = smem_layout(bins.n_bins, n_k, rdf, qa.stage_cap).total;
  if (n_k > 0 || rdf) {
    rc = rdf ? dispatch_k<true>(g, qa, smem, s) : dispatch_k<false>(g, qa, smem, s);
    if (rc) return rc;
  }
  k_query_epilogue<<<1, 32, 0, s>>>(g->nbr.geo, g->ctr.geo, d_meta);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
