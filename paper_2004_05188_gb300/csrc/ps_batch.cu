// Batched sweeps: many ROIs and a parameter sweep per ROI in one persistent launch.
//
// The paper's batch queue takes an a-priori list of (statistic, ion-type
// combination, dataset) tasks and evaluates all of them per ROI from one
// neighbour search (Suppl. "Customized user defined batch processing queues"),
// to support parameter-sensitivity studies over many specimens (Results,
// application to experimental datasets).  Here one enumeration per (ROI, cell
// batch) at the largest r_max serves every sweep point exactly:
//   - every k = 1..k_max comes from the per-lane sorted top-k lists (one list per
//     distinct neighbour type set);
//   - every smaller r_max is a prefix of the histograms (the bin edges coincide),
//     and a k-th distance beyond a smaller r_max is "not found" there;
//   - every d_srf threshold t_q is a suffix sum over d_srf classes
//     [t_c, t_{c+1}) accumulated separately;
//   - every type pair comes from the same enumeration (the record carries the
//     ion type; a hit counts for the pairs whose central and neighbour sets hold
//     both ends).
// Work: one queue over all ROIs, items (cell, <= 32 centrals) in ROI order,
// padded per ROI to whole chunks of 8 so a CTA (8 warps) always works on one
// ROI and can keep that ROI's RDF counts in shared memory.  kNN counts go to
// global memory (one update per central, k and pair).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ps_internal.cuh"

namespace ps {

constexpr int kChunk = 8;        // items per CTA fetch (one per warp)
constexpr int kBatchRuns = 25;

struct BRoi {
  const float4* nrec;
  const uint32_t* nstart;
  const Geo* ngeo;
  const float4* crec;
  const uint32_t* cstart;
  const uint2* witem;
  const Geo* cgeo;
  const float* dsrf;
  uint32_t cap;  // capacity of witem
};

struct BatchArgs {
  const BRoi* roi;
  const uint32_t* item_off;  // [n_roi + 1] padded exclusive prefix of the ROIs' item counts
  uint32_t n_roi;
  uint32_t* next;            // work counter (chunks of kChunk items)
  int stencil;
  double r0, dr;
  uint32_t n_bins;           // bins at the largest r_max
  uint32_t n_pairs, n_cls, k_max;
  uint32_t n_lists;
  uint32_t list_of[4];       // pair -> top-k list
  uint64_t ctr_mask[4][4];
  uint64_t nbr_mask[4][4];
  uint64_t list_mask[2][4];  // neighbour set of each list
  float cls_min[4];          // d_srf class lower bounds (ascending)
  unsigned long long* acc;   // per ROI accumulators, acc_len each
  uint32_t acc_len;
};

// accumulator layout of one ROI: for each (pair p, class c) a block of
//   rdf[n_bins] | rdf_below | n_central | knn[k_max][n_bins] | knn_below[k_max]
__host__ __device__ inline uint32_t acc_block(uint32_t nb, uint32_t kmax) { return nb + 2 + kmax * nb + kmax; }

__device__ __forceinline__ bool mask_has(const uint64_t* m, uint32_t t) { return (m[t >> 6] >> (t & 63)) & 1ull; }

template <int K>
__device__ __forceinline__ void tk_insert(float (&top)[K], float x) {
  if (x < top[K - 1]) {
#pragma unroll
    for (int t = K - 1; t > 0; --t) top[t] = fminf(top[t], fmaxf(x, top[t - 1]));
    top[0] = fminf(top[0], x);
  }
}

template <int K>
__device__ __forceinline__ float tk_get(const float (&top)[K], uint32_t idx) {
  float v = INFINITY;
#pragma unroll
  for (int t = 0; t < K; ++t)
    if ((uint32_t)t == idx) v = top[t];
  return v;
}

__device__ __forceinline__ uint32_t bbin(float d2, const float* sE, uint32_t nb, float r0f, float inv_dr) {
  const float d = d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
  int b = (int)((d - r0f) * inv_dr);
  b = b < 0 ? 0 : (b >= (int)nb ? (int)nb - 1 : b);
  if (d2 < sE[b] || d2 >= sE[b + 1]) {
    while (b > 0 && d2 < sE[b]) --b;
    while (b + 1 < (int)nb && d2 >= sE[b + 1]) ++b;
  }
  return (uint32_t)b;
}

template <int KMAX, int NL>
__global__ void __launch_bounds__(256, 3) k_batch_query(const BatchArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_buf[8][32];
  __shared__ float s_hd[8][512];
  __shared__ uint32_t s_ht[8][512];
  __shared__ uint32_t s_rsrc[8][kBatchRuns], s_rpre[8][kBatchRuns + 1];
  __shared__ uint32_t s_chunk, s_roi;
  __shared__ uint32_t s_tinfo[256];  // per type: bit l = in list l's neighbour set, bit 2 + p = in pair p's

  const uint32_t nb = a.n_bins, P = a.n_pairs, C = a.n_cls;
  // 64-bit pair counters (a CTA may count more than 2^32 pairs of one ROI), 32-bit central counts
  float* sE = reinterpret_cast<float*>(smem);
  unsigned long long* s_rdf = reinterpret_cast<unsigned long long*>(smem + ((nb + 1) * 4 + 15) / 16 * 16);  // [P][C][nb+1]
  uint32_t* s_nc = reinterpret_cast<uint32_t*>(s_rdf + P * C * (nb + 1));                                   // [P][C]
  const uint32_t n_rdf = P * C * (nb + 1);  // per (p, c): nb bins then the below-range count
  for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) {
    const double e = __dadd_rn(a.r0, __dmul_rn((double)b, a.dr));
    sE[b] = __double2float_rn(__dmul_rn(e, e));
  }
  for (uint32_t i = threadIdx.x; i < n_rdf; i += blockDim.x) s_rdf[i] = 0ull;
  for (uint32_t i = threadIdx.x; i < P * C; i += blockDim.x) s_nc[i] = 0;
  for (uint32_t t = threadIdx.x; t < 256; t += blockDim.x) {
    uint32_t v = 0;
    for (uint32_t l = 0; l < (uint32_t)NL; ++l) v |= (mask_has(a.list_mask[l], t) ? 1u : 0u) << l;
    for (uint32_t pp = 0; pp < P; ++pp) v |= (mask_has(a.nbr_mask[pp], t) ? 1u : 0u) << (2 + pp);
    s_tinfo[t] = v;
  }
  __syncthreads();
  const float Emax = sE[nb], E0 = sE[0], r0f = (float)a.r0, inv_dr = (float)(1.0 / a.dr);
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t total = a.item_off[a.n_roi];
  const uint32_t blk = acc_block(nb, a.k_max);
  int cur = -1;

  auto flush = [&](int roi) {
    __syncthreads();
    unsigned long long* A = a.acc + (size_t)roi * a.acc_len;
    for (uint32_t i = threadIdx.x; i < n_rdf; i += blockDim.x) {
      const unsigned long long v = s_rdf[i];
      if (!v) continue;
      // rdf[b] at offset b of block pc, the below-range count at offset nb
      atomicAdd(&A[(i / (nb + 1)) * blk + i % (nb + 1)], v);
      s_rdf[i] = 0ull;
    }
    for (uint32_t i = threadIdx.x; i < P * C; i += blockDim.x) {
      if (s_nc[i]) atomicAdd(&A[i * blk + nb + 1], (unsigned long long)s_nc[i]);
      s_nc[i] = 0;
    }
    __syncthreads();
  };

  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t ch = atomicAdd(a.next, (uint32_t)kChunk);
      s_chunk = ch;
      uint32_t lo = 0, hi = a.n_roi;  // item_off[lo] <= ch < item_off[hi]
      if (ch < total)
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (a.item_off[mid] <= ch)
            lo = mid;
          else
            hi = mid;
        }
      s_roi = lo;
    }
    __syncthreads();
    const uint32_t chunk = s_chunk, roi = s_roi;
    if (chunk >= total) break;
    if ((int)roi != cur) {
      if (cur >= 0) flush(cur);
      cur = (int)roi;
    }
    const BRoi R = a.roi[roi];
    const uint32_t l_item = chunk + w - a.item_off[roi];
    const uint32_t n_front = R.cgeo->work_n2, n_items = n_front + R.cgeo->work_n3;
    unsigned long long* A = a.acc + (size_t)roi * a.acc_len;
    if (l_item < n_items) {
      const Geo ng = *R.ngeo;
      const uint2 it = work_item(R.witem, R.cap, n_front, l_item);
      const uint32_t c = it.x, first = it.y >> 6, cnt = it.y & 63u;
      const uint32_t c0 = R.cstart[c] + first;
      // run table
      uint32_t src = 0, len = 0;
      {
        const int s = a.stencil, wd = 2 * s + 1;
        const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
        const int y = (int)cy + (int)(lane % wd) - s, z = (int)cz + (int)(lane / wd) - s;
        if ((int)lane < wd * wd && y >= 0 && z >= 0 && y < (int)ng.dims[1] && z < (int)ng.dims[2]) {
          const uint32_t xlo = cx >= (uint32_t)s ? cx - s : 0;
          const uint32_t xhi = cx + s < ng.dims[0] ? cx + s : ng.dims[0] - 1;
          const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
          src = R.nstart[row + xlo];
          len = R.nstart[row + xhi + 1] - src;
        }
      }
      uint32_t pre = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= (uint32_t)o) pre += y;
      }
      const uint32_t n_cand = __shfl_sync(0xffffffffu, pre, 31);
      uint32_t* rsrc = s_rsrc[w];
      uint32_t* rpre = s_rpre[w];
      __syncwarp();
      if (lane < (uint32_t)kBatchRuns) {
        rsrc[lane] = src;
        rpre[lane + 1] = pre;
      }
      if (lane == 0) rpre[0] = 0;
      __syncwarp();

      // this lane's central: type, class, pair membership
      const bool valid = lane < cnt;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      uint32_t pw = ~0u, cls = 0, pmask = 0;
      if (valid) {
        p = R.crec[c0 + lane];
        pw = __float_as_uint(p.w);
        const uint32_t ti = pw & 0xFFu;
        const float di = R.dsrf ? R.dsrf[pw >> 8] : INFINITY;
        for (uint32_t q = 1; q < C; ++q)
          if (di >= a.cls_min[q]) cls = q;
        for (uint32_t pp = 0; pp < P; ++pp)
          if (mask_has(a.ctr_mask[pp], ti)) pmask |= 1u << pp;
      }
      const float emax = valid ? Emax : -INFINITY;
      const uint32_t lt = (1u << lane) - 1u;
      float top[NL][KMAX];
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int t = 0; t < KMAX; ++t) top[l][t] = INFINITY;
      const unsigned long long px = f2_pack(p.x, p.x), py = f2_pack(p.y, p.y), pz = f2_pack(p.z, p.z);
      float* hd = s_hd[w];
      uint32_t* ht = s_ht[w];
      float* bf = reinterpret_cast<float*>(s_buf[w]);
      int rr = 0;
      auto fetch = [&](uint32_t pos) -> float4 {
        if (pos >= n_cand) return make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(~0u));
        while (pos >= rpre[rr + 1]) ++rr;
        return __ldg(R.nrec + rsrc[rr] + (pos - rpre[rr]));
      };
      float4 nxt = fetch(lane);
      for (uint32_t b0 = 0; b0 < n_cand; b0 += 32) {
        __syncwarp();
        {
          float* d = bf + (lane >> 1) * 8 + (lane & 1);
          d[0] = nxt.x, d[2] = nxt.y, d[4] = nxt.z, d[6] = nxt.w;
        }
        __syncwarp();
        nxt = fetch(b0 + 32 + lane);
        for (int half = 0; half < 2; ++half) {
          uint32_t nh = 0;
#pragma unroll 2
          for (int t = half * 8; t < half * 8 + 8; ++t) {
            const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(bf)[2 * t];
            const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(bf)[2 * t + 1];
            float d2v[2], wv[2];
            dist2_x2(px, py, pz, xy.x, xy.y, zw.x, d2v[0], d2v[1]);
            f2_unpack(zw.y, wv[0], wv[1]);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const uint32_t qw = __float_as_uint(wv[e]);
              const bool hit = d2v[e] < emax && qw != pw;
              uint32_t tag = 0;
              if (hit) {
                const uint32_t ti = s_tinfo[qw & 0xFFu];
#pragma unroll
                for (int l = 0; l < NL; ++l)
                  if (((ti >> l) & 1u) && d2v[e] < top[l][KMAX - 1]) tk_insert(top[l], d2v[e]);
                tag = (ti >> 2) & pmask;
              }
              const bool rec = tag != 0;
              const uint32_t bal = __ballot_sync(0xffffffffu, rec);
              if (rec) {
                const uint32_t slot = nh + __popc(bal & lt);
                hd[slot] = d2v[e];
                ht[slot] = tag | (cls << 8);
              }
              nh += __popc(bal);
            }
          }
          __syncwarp();
          for (uint32_t h = lane; h < nh; h += 32) {
            const float d2 = hd[h];
            const uint32_t tg = ht[h], cc = tg >> 8;
            const bool below = d2 < E0;
            const uint32_t bn = below ? 0u : bbin(d2, sE, nb, r0f, inv_dr);
            for (uint32_t pp = 0; pp < P; ++pp) {
              if (!((tg >> pp) & 1u)) continue;
              atomicAdd(&s_rdf[(pp * C + cc) * (nb + 1) + (below ? nb : bn)], 1ull);
            }
          }
          __syncwarp();
        }
      }
      // per central: counts and the k-th distances of every pair
      if (valid) {
        for (uint32_t pp = 0; pp < P; ++pp) {
          if (!((pmask >> pp) & 1u)) continue;
          const uint32_t pc = pp * C + cls;
          atomicAdd(&s_nc[pc], 1u);
          const uint32_t l = a.list_of[pp];
          for (uint32_t k = 0; k < a.k_max; ++k) {
            float D = INFINITY;
#pragma unroll
            for (int ll = 0; ll < NL; ++ll)
              if ((uint32_t)ll == l) D = tk_get(top[ll], k);
            if (!(D < Emax)) continue;  // not found: derived from the counts
            if (D < E0)
              atomicAdd(&A[pc * blk + nb + 2 + a.k_max * nb + k], 1ull);
            else
              atomicAdd(&A[pc * blk + nb + 2 + k * nb + bbin(D, sE, nb, r0f, inv_dr)], 1ull);
          }
        }
      }
    }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

// Padded item offsets: item_off[r] = sum over ROIs before r of ceil(items / kChunk) * kChunk.
__global__ void k_batch_offsets(const BRoi* __restrict__ roi, uint32_t n_roi, uint32_t* __restrict__ item_off,
                                uint32_t* __restrict__ next) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t r = 0; r < n_roi; ++r) {
      item_off[r] = acc;
      const uint32_t n = roi[r].cgeo->work_n2 + roi[r].cgeo->work_n3;
      acc += (n + kChunk - 1) / kChunk * kChunk;
    }
    item_off[n_roi] = acc;
    *next = 0;
  }
}

// Expands the class accumulators into one result per (ROI, pair, r_max, d_srf threshold),
// in the layout of ps_spatstat: rdf[n_bins] | knn[k_max][n_bins] | meta[PS_META_LEN(k_max)].
__global__ void __launch_bounds__(256) k_batch_expand(const unsigned long long* __restrict__ acc, uint32_t acc_len,
                                                      uint32_t nb, uint32_t P, uint32_t C, uint32_t kmax, uint32_t R,
                                                      const uint32_t* __restrict__ rbins, unsigned long long* out) {
  griddep_wait();
  griddep_launch();
  const uint32_t rec = nb + kmax * nb + PS_META_LEN(kmax);
  const uint32_t blk = acc_block(nb, kmax);
  const uint32_t id = blockIdx.x;  // ((roi * P + p) * R + r) * C + q
  const uint32_t q = id % C, r = (id / C) % R, pp = (id / (C * R)) % P, roi = id / (C * R * P);
  const unsigned long long* A = acc + (size_t)roi * acc_len + (size_t)pp * C * blk;
  unsigned long long* O = out + (size_t)id * rec;
  const uint32_t nbr_ = rbins[r];
  __shared__ unsigned long long s_red[8];
  // rdf
  unsigned long long binned = 0;
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    unsigned long long v = 0;
    if (b < nbr_)
      for (uint32_t c = q; c < C; ++c) v += A[c * blk + b];
    O[b] = v;
    binned += v;
  }
  // knn
  for (uint32_t i = threadIdx.x; i < kmax * nb; i += blockDim.x) {
    const uint32_t k = i / nb, b = i % nb;
    unsigned long long v = 0;
    if (b < nbr_)
      for (uint32_t c = q; c < C; ++c) v += A[c * blk + nb + 2 + k * nb + b];
    O[nb + i] = v;
  }
  for (int o = 16; o > 0; o >>= 1) binned += __shfl_xor_sync(0xffffffffu, binned, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = binned;
  __syncthreads();
  unsigned long long* M = O + nb + kmax * nb;
  if (threadIdx.x == 0) {
    unsigned long long tb = 0, nc = 0, below = 0;
    for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) tb += s_red[i];
    for (uint32_t c = q; c < C; ++c) nc += A[c * blk + nb + 1], below += A[c * blk + nb];
    M[PS_META_N_CENTRAL] = nc;
    M[PS_META_N_PAIRS] = tb;
    M[PS_META_N_BELOW] = below;
    M[PS_META_STATUS] = 0;
  }
  // per k: not found = centrals - found in range - below range
  for (uint32_t k = threadIdx.x; k < kmax; k += blockDim.x) {
    unsigned long long nc = 0, found = 0, kb = 0;
    for (uint32_t c = q; c < C; ++c) {
      nc += A[c * blk + nb + 1];
      kb += A[c * blk + nb + 2 + kmax * nb + k];
      for (uint32_t b = 0; b < nbr_; ++b) found += A[c * blk + nb + 2 + k * nb + b];
    }
    M[PS_META_HEAD + 2 * k] = nc - found - kb;
    M[PS_META_HEAD + 2 * k + 1] = kb;
  }
}

}  // namespace ps

struct ps_batch {
  ps_sweep sw;
  std::vector<ps_dataset> ds;
  std::vector<ps_grid*> grids;
  ps::BRoi* d_roi = nullptr;
  uint32_t* d_item_off = nullptr;
  uint32_t* d_next = nullptr;
  uint32_t* d_rbins = nullptr;
  unsigned long long* d_acc = nullptr;
  uint32_t acc_len = 0, n_lists = 0, list_of[4] = {0, 0, 0, 0};
  uint64_t list_mask[2][4];
  uint64_t nbr_union[4], ctr_union[4];
  float r_cut = 0.f;
};

using namespace ps;

template <int KMAX, int NL>
static int launch_batch(const ps_batch* b, const BatchArgs& a, uint32_t smem, int sms, cudaStream_t st) {
  auto kern = k_batch_query<KMAX, NL>;
  PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
  if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "batched query kernel does not fit on an SM");
  PS_LAUNCH(PS_KID_BATCH, st, PS_CUDA(launch_pdl(kern, sms * per_sm, 256, smem, st, a)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}


extern "C" {

int ps_batch_create(const ps_dataset* ds, int n_ds, const ps_sweep* sw, ps_batch** out) {
  if (!out || !ds || !sw || n_ds < 1) return fail(PS_ERR_INVALID_ARG, "ps_batch_create: NULL argument or n_ds < 1");
  *out = nullptr;
  if (sw->struct_size < sizeof(ps_sweep)) return fail(PS_ERR_INVALID_ARG, "ps_batch_create: sweep struct_size");
  const ps_sweep& s = *sw;
  if (!(s.bins.dr > 0.0) || !(s.bins.r0 >= 0.0) || s.bins.n_bins < 1 || s.bins.n_bins > 512)
    return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: need dr > 0, r0 >= 0 and 1..512 bins");
  if (s.n_rmax < 1 || s.n_rmax > 4 || s.n_dsrf < 1 || s.n_dsrf > 4 || s.n_pairs < 1 || s.n_pairs > 4)
    return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: 1..4 r_max values, d_srf thresholds and type pairs");
  if (s.k_max < 1 || s.k_max > PS_K_MAX) return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: k_max in 1..32");
  for (uint32_t r = 0; r < s.n_rmax; ++r)
    if (s.rmax_bins[r] < 1 || s.rmax_bins[r] > s.bins.n_bins || (r && s.rmax_bins[r] <= s.rmax_bins[r - 1]))
      return fail(PS_ERR_INVALID_ARG, "ps_batch_create: rmax_bins must ascend within 1..n_bins");
  if (s.rmax_bins[s.n_rmax - 1] != s.bins.n_bins)
    return fail(PS_ERR_INVALID_ARG, "ps_batch_create: the last r_max must be bins.n_bins");
  for (uint32_t q = 0; q < s.n_dsrf; ++q)
    if (std::isnan(s.dsrf_min[q]) || (q && !(s.dsrf_min[q] > s.dsrf_min[q - 1])))
      return fail(PS_ERR_INVALID_ARG, "ps_batch_create: dsrf_min must ascend");
  if (s.cell_scale != 0.0f && !(s.cell_scale >= 0.5f))
    return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: cell_scale must be 0 (default) or >= 0.5");
  const uint32_t smem_rdf = s.n_pairs * s.n_dsrf * s.bins.n_bins;
  if (smem_rdf > 8192) return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: pairs x thresholds x bins > 8192");
  ps_batch* b = new (std::nothrow) ps_batch();
  if (!b) return fail(PS_ERR_OOM, "host allocation failed");
  b->sw = s;
  // distinct neighbour sets -> top-k lists
  for (uint32_t p = 0; p < s.n_pairs; ++p) {
    int found = -1;
    for (uint32_t l = 0; l < b->n_lists; ++l)
      if (!memcmp(b->list_mask[l], s.nbr_mask[p], sizeof(uint64_t) * 4)) found = (int)l;
    if (found < 0) {
      if (b->n_lists == 2) {
        delete b;
        return fail(PS_ERR_UNSUPPORTED, "ps_batch_create: at most 2 distinct neighbour type sets");
      }
      memcpy(b->list_mask[b->n_lists], s.nbr_mask[p], sizeof(uint64_t) * 4);
      found = (int)b->n_lists++;
    }
    b->list_of[p] = (uint32_t)found;
  }
  for (int w = 0; w < 4; ++w) {
    b->nbr_union[w] = b->ctr_union[w] = 0;
    for (uint32_t p = 0; p < s.n_pairs; ++p) b->nbr_union[w] |= s.nbr_mask[p][w], b->ctr_union[w] |= s.ctr_mask[p][w];
  }
  const double stop = s.bins.r0 + (double)s.bins.n_bins * s.bins.dr;
  b->r_cut = (float)(stop * (1.0 + 1e-6));
  b->acc_len = s.n_pairs * s.n_dsrf * acc_block(s.bins.n_bins, s.k_max);
  ps_grid_opts go;
  memset(&go, 0, sizeof(go));
  go.struct_size = sizeof(go);
  go.cell_scale = s.cell_scale;
  int rc = PS_OK;
  for (int i = 0; i < n_ds && rc == PS_OK; ++i) {
    if (ds[i].n < 0 || ds[i].n >= (1 << 24)) rc = fail(PS_ERR_UNSUPPORTED, "ps_batch_create: ROIs hold < 2^24 ions");
    if (rc == PS_OK && ds[i].n > 0 && (!ds[i].xyz || !ds[i].type))
      rc = fail(PS_ERR_INVALID_ARG, "ps_batch_create: dataset xyz/type is NULL");
    if (rc) break;
    b->ds.push_back(ds[i]);
    ps_grid* g = nullptr;
    rc = ps_grid_create(ds[i].n, &go, &g);
    if (rc == PS_OK) {
      g->pack_type = true;
      b->grids.push_back(g);
    }
  }
  auto cleanup = [&](int code) {
    for (ps_grid* g : b->grids) ps_grid_destroy(g);
    dev_free(b->d_roi);
    dev_free(b->d_item_off);
    dev_free(b->d_next);
    dev_free(b->d_rbins);
    dev_free(b->d_acc);
    delete b;
    return code;
  };
  if (rc) return cleanup(rc);
  cudaError_t e = dev_malloc((void**)&b->d_roi, sizeof(BRoi) * n_ds);
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_item_off, sizeof(uint32_t) * (n_ds + 1));
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_next, sizeof(uint32_t));
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_rbins, sizeof(uint32_t) * 4);
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_acc, sizeof(unsigned long long) * (size_t)b->acc_len * n_ds);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(batch)"));
  std::vector<BRoi> h(n_ds);
  for (int i = 0; i < n_ds; ++i) {
    ps_grid* g = b->grids[i];
    h[i] = BRoi{g->nbr.rec, g->nbr.start, g->nbr.geo, g->ctr.rec,       g->ctr.start,
                g->ctr.witem, g->ctr.geo,  ds[i].dsrf, g->item_cap};
  }
  e = cudaMemcpy(b->d_roi, h.data(), sizeof(BRoi) * n_ds, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_rbins, s.rmax_bins, sizeof(uint32_t) * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMemcpy(batch)"));
  *out = b;
  return PS_OK;
}

int ps_batch_destroy(ps_batch* b) {
  if (!b) return PS_OK;
  cudaDeviceSynchronize();
  for (ps_grid* g : b->grids) ps_grid_destroy(g);
  dev_free(b->d_roi);
  dev_free(b->d_item_off);
  dev_free(b->d_next);
  dev_free(b->d_rbins);
  dev_free(b->d_acc);
  delete b;
  return PS_OK;
}

int64_t ps_batch_out_len(const ps_batch* b) {
  if (!b) return -1;
  const ps_sweep& s = b->sw;
  const int64_t rec = s.bins.n_bins + (int64_t)s.k_max * s.bins.n_bins + PS_META_LEN(s.k_max);
  return (int64_t)b->ds.size() * s.n_pairs * s.n_rmax * s.n_dsrf * rec;
}

int ps_batch_run(ps_batch* b, uint64_t* d_out, void* stream) {
  if (!b || !d_out) return fail(PS_ERR_INVALID_ARG, "ps_batch_run: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ps_sweep& s = b->sw;
  const uint32_t n_roi = (uint32_t)b->ds.size();
  // grids and central lists of every ROI (records carry the ion type)
  for (uint32_t i = 0; i < n_roi; ++i) {
    int rc = ps_grid_build(b->grids[i], b->ds[i].xyz, b->ds[i].type, b->ds[i].n, b->nbr_union, b->r_cut, stream);
    if (rc) return rc;
    rc = build_central_list(b->grids[i], b->ds[i].dsrf, b->ctr_union, s.dsrf_min[0], st);
    if (rc) return rc;
  }
  PS_CUDA(cudaMemsetAsync(b->d_acc, 0, sizeof(unsigned long long) * (size_t)b->acc_len * n_roi, st));
  PS_LAUNCH(PS_KID_BATCH, st, PS_CUDA(launch_pdl(k_batch_offsets, 1, 32, 0, st, b->d_roi, n_roi, b->d_item_off, b->d_next)));
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.roi = b->d_roi;
  a.item_off = b->d_item_off;
  a.n_roi = n_roi;
  a.next = b->d_next;
  a.stencil = b->grids[0]->stencil;
  a.r0 = s.bins.r0;
  a.dr = s.bins.dr;
  a.n_bins = s.bins.n_bins;
  a.n_pairs = s.n_pairs;
  a.n_cls = s.n_dsrf;
  a.k_max = s.k_max;
  a.n_lists = b->n_lists;
  for (uint32_t p = 0; p < s.n_pairs; ++p) {
    a.list_of[p] = b->list_of[p];
    for (int w = 0; w < 4; ++w) a.ctr_mask[p][w] = s.ctr_mask[p][w], a.nbr_mask[p][w] = s.nbr_mask[p][w];
  }
  for (uint32_t l = 0; l < b->n_lists; ++l)
    for (int w = 0; w < 4; ++w) a.list_mask[l][w] = b->list_mask[l][w];
  for (uint32_t q = 0; q < s.n_dsrf; ++q) a.cls_min[q] = s.dsrf_min[q];
  a.acc = b->d_acc;
  a.acc_len = b->acc_len;
  const uint32_t smem = ((s.bins.n_bins + 1) * 4 + 15) / 16 * 16 + s.n_pairs * s.n_dsrf * ((s.bins.n_bins + 1) * 8 + 4);
  const int sms = b->grids[0]->num_sms;
  int rc;
  const uint32_t k = s.k_max;
  if (b->n_lists == 1)
    rc = k <= 8 ? launch_batch<8, 1>(b, a, smem, sms, st)
         : k <= 16 ? launch_batch<16, 1>(b, a, smem, sms, st)
         : k <= 20 ? launch_batch<20, 1>(b, a, smem, sms, st)
                   : launch_batch<32, 1>(b, a, smem, sms, st);
  else
    rc = k <= 8 ? launch_batch<8, 2>(b, a, smem, sms, st)
         : k <= 16 ? launch_batch<16, 2>(b, a, smem, sms, st)
         : k <= 20 ? launch_batch<20, 2>(b, a, smem, sms, st)
                   : launch_batch<32, 2>(b, a, smem, sms, st);
  if (rc) return rc;
  const uint32_t n_out = n_roi * s.n_pairs * s.n_rmax * s.n_dsrf;
  PS_LAUNCH(PS_KID_BATCH, st,
            PS_CUDA(launch_pdl(k_batch_expand, n_out, 256, 0, st, b->d_acc, b->acc_len, s.bins.n_bins, s.n_pairs, s.n_dsrf, s.k_max,
                                                  s.n_rmax, b->d_rbins, reinterpret_cast<unsigned long long*>(d_out))));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // extern "C"
