// Exact kNN + RDF query over the cell grid.
//
// The paper evaluates one spherical ROI per central ion and machines the ROIs
// off with a dynamic schedule, each thread keeping its own result buffers that
// are merged afterwards (Suppl. "Customized user defined batch processing
// queues").  Here the ROIs of one cell of the grid share their candidates: the
// cells within `stencil` cells of it (27 cells for cells of edge >= r_cut, 125
// for cells of edge >= r_cut/2, up to 343 for r_cut/3, less the cells that
// cannot hold a pair within r_cut), read as x-contiguous runs of sorted records.
// Two persistent kernels take work from device counters (the dynamic
// schedule):
//
//   warp kernel  heavy items = (cell with >= 16 centrals, batch of <= 32 of
//                them): the candidates are read 32 at a time with one coalesced
//                load into a per-warp shared buffer (the next batch is
//                prefetched into registers meanwhile); each lane holds one
//                central and walks the buffer (shared-memory broadcast).
//                Light items (sparser cells) are taken 32 at a time and each of
//                their centrals gets one thread that walks its own stencil.
//   CTA kernel   for cells with >= dense_min centrals (an option): one CTA per
//                cell; the runs are staged into shared memory with bulk
//                asynchronous copies (cp.async.bulk, completion on an mbarrier)
//                and one thread per central walks them.
//
// Each thread keeps the k smallest squared distances in registers (sorted
// insertion).  Counts go to per-CTA shared-memory histograms (the per-thread
// buffers) added to the uint64 global histograms when the CTA finishes.
//
// The query in passes (ps_grid_opts.split) reuses the warp kernel for its near
// kNN pass (vertex mode: the centrals sorted by the vertex-centred grid, each
// item against the 2 x 2 x 2 cells around its vertex) and adds k_knn_list (the
// full-radius kNN of the centrals that pass lists) and k_rdf_sym (the RDF over
// unordered pairs of neighbour records).
#include <cstring>
#include <vector>

#include "ps_internal.cuh"

namespace ps {

constexpr int kMaxRuns = 49;  // (2 * stencil + 1)^2 for stencil <= 3

struct QueryArgs {
  const float4* nrec;
  const uint32_t* nstart;
  const Geo* ngeo;
  const float4* crec;
  const uint32_t* cstart;
  const uint32_t* cwork;
  const uint2* witem;
  const uint2* whi;   // very heavy items (taken before those of witem)
  uint32_t work_cap;  // capacity of witem (light items grow from its end)
  Geo* cgeo;
  int stencil;
  double r0, dr;
  uint32_t n_bins;
  uint32_t n_k;
  uint32_t k_need;     // max requested k
  uint32_t stage_cap;  // float4 records per staging chunk (CTA kernel)
  uint32_t ks[PS_MAX_KLIST];
  uint64_t* rdf;
  uint64_t* knn;
  uint64_t* meta;
  float* kth;
  uint32_t* nwithin;
  int64_t n;  // ions in the cloud (stride of kth)
  // passes of the split query (zero / null for the combined one)
  float emax_near;        // > 0: kNN within this squared range only; a central with fewer than k_need
                          // neighbours there is marked in need[] instead of being counted
  uint32_t* need;         // per central record: 1 = needs the full-radius search (near pass writes it)
  int fallback;           // 1: only the centrals marked in need[] (the full-radius kNN pass)
  uint32_t* next_front;   // work counters of the front (heavy) and back (light) items
  uint32_t* next_light;
  const uint32_t* pfx;    // symmetric RDF pass: central prefix over the neighbour records
  int vertex;             // near kNN pass on the vertex-centred central list (see vertex_run)
  // bin lookup table (lut_shift = 0: none): cell c covers the float32 bit patterns
  // [(lut_base + c) << lut_shift, (lut_base + c + 1) << lut_shift), at most one interior edge each
  uint32_t lut_shift, lut_base, lut_n;
  // half-width of each stencil row (dy, dz), at [(dz + s) (2s + 1) + dy + s]: the row's cells
  // cx - w .. cx + w can hold a record within r_cut of the cell's records, the others cannot
  // (-1: none); w = s unless the cell is small against r_cut (see row_widths)
  int8_t row_w[kMaxRuns];
};

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

// bin b in [0, nb) with sE[b] <= d2 < sE[b+1]; caller guarantees sE[0] <= d2 < sE[nb].
// The guess from an approximate square root is checked against the exact edge
// table; the (rare) wrong guess is walked to the right bin.
__device__ __forceinline__ uint32_t bin_index(float d2, const float* sE, uint32_t nb, float r0f, float inv_dr) {
  const float d = d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
  int b = (int)((d - r0f) * inv_dr);
  b = b < 0 ? 0 : (b >= (int)nb ? (int)nb - 1 : b);
  if (d2 < sE[b] || d2 >= sE[b + 1]) {
    while (b > 0 && d2 < sE[b]) --b;
    while (b + 1 < (int)nb && d2 >= sE[b + 1]) ++b;
  }
  return (uint32_t)b;
}

struct SmemLayout {
  uint32_t off_E, off_lut, off_rdf, off_knn, off_kmeta, off_stage, total;
  bool priv;
};

constexpr uint32_t kLutMax = 4096;  // entries of the bin lookup table (uint32)

constexpr uint32_t kPrivBins = 512;  // up to this many bins each warp keeps its own 32-bit RDF row

__host__ __device__ inline SmemLayout smem_layout(uint32_t n_bins, uint32_t n_k, bool rdf, uint32_t stage_cap,
                                                  bool allow_priv = false, uint32_t lut_n = 0) {
  SmemLayout L;
  uint32_t o = 0;
  L.priv = allow_priv && rdf && n_bins <= kPrivBins;
  L.off_E = o;
  o += (n_bins + 1) * 4;
  L.off_lut = o;
  o += rdf ? lut_n * 4 : 0;
  o = (o + 7u) & ~7u;
  L.off_rdf = o;
  o += rdf ? (L.priv ? 8 * n_bins * 4 : n_bins * 8) : 0;
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

// Per-CTA result buffers in shared memory.
template <bool RDF>
struct Hist {
  float* sE;
  unsigned long long* s_rdf;  // CTA row, 64-bit: per-CTA pair counts can pass 2^32 on large clouds
  uint32_t* s_rdfw;           // or one 32-bit row per warp (priv), flushed by its warp before it could wrap
  bool priv;
  uint32_t* s_knn;            // per-CTA central counts stay below n < 2^32
  uint32_t* s_kmeta;
  uint32_t* lut;              // bin lookup table (see QueryArgs)
  uint32_t lut_shift, lut_base, lut_mask;
  float Emax, E0, r0f, inv_dr;
  uint32_t nb;

  __device__ void init(const QueryArgs& a, unsigned char* smem, uint32_t stage_cap, bool allow_priv = false) {
    const SmemLayout L = smem_layout(a.n_bins, a.n_k, RDF, stage_cap, allow_priv, a.lut_n);
    sE = reinterpret_cast<float*>(smem + L.off_E);
    lut = reinterpret_cast<uint32_t*>(smem + L.off_lut);
    lut_shift = RDF ? a.lut_shift : 0u;
    lut_base = a.lut_base;
    lut_mask = (1u << lut_shift) - 1u;
    priv = L.priv;
    s_rdf = reinterpret_cast<unsigned long long*>(smem + L.off_rdf);
    s_rdfw = reinterpret_cast<uint32_t*>(smem + L.off_rdf) + (threadIdx.x >> 5) * a.n_bins;
    s_knn = reinterpret_cast<uint32_t*>(smem + L.off_knn);
    s_kmeta = reinterpret_cast<uint32_t*>(smem + L.off_kmeta);
    nb = a.n_bins;
    // edge table: the same double formula as the host, E[b] = (float)((r0 + b*dr)^2)
    for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) {
      const double e = __dadd_rn(a.r0, __dmul_rn((double)b, a.dr));
      sE[b] = __double2float_rn(__dmul_rn(e, e));
    }
    if (RDF) {
      if (priv)
        for (uint32_t b = threadIdx.x; b < 8 * nb; b += blockDim.x) reinterpret_cast<uint32_t*>(s_rdf)[b] = 0;
      else
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) s_rdf[b] = 0ull;
    }
    for (uint32_t b = threadIdx.x; b < a.n_k * nb; b += blockDim.x) s_knn[b] = 0;
    for (uint32_t b = threadIdx.x; b < 2 * a.n_k; b += blockDim.x) s_kmeta[b] = 0;
    __syncthreads();
    if (RDF && lut_shift) {
      // entry c = b0 << 17 | off: b0 the largest b < nb with E[b] <= the smallest value of cell c
      // (0 below E[0]); off the low lut_shift bits of the next interior edge E[b0 + 1] if it lies
      // in the cell (at most one does), else 2^16, above every low part
      for (uint32_t c = threadIdx.x; c < a.lut_n; c += blockDim.x) {
        const uint32_t c0 = (lut_base + c) << lut_shift;
        const float v = __uint_as_float(c0);
        uint32_t lo = 0, hi = nb;  // invariant: E[lo] <= v or lo == 0; E[hi] > v or hi == nb
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (sE[mid] <= v)
            lo = mid;
          else
            hi = mid;
        }
        uint32_t off = 1u << 16;
        if (lo + 1 < nb) {
          const uint32_t e = __float_as_uint(sE[lo + 1]);
          if (e >= c0 && e - c0 <= lut_mask) off = e & lut_mask;
        }
        lut[c] = lo << 17 | off;
      }
      __syncthreads();
    }
    Emax = sE[nb];
    E0 = sE[0];
    r0f = (float)a.r0;
    inv_dr = (float)(1.0 / a.dr);
  }

  // bin b in [0, nb) with E[b] <= d2 < E[b+1] for E[0] <= d2 < E[nb]: from the lookup table (the
  // cell of d2's bit pattern holds at most one interior edge, so the bin is the entry or the next
  // one), else from an approximate square root checked against the edges
  // (d2 >= 0 below E[nb]; the table's first cell lies wholly below E[1], so values below the
  // table take its entry, bin 0)
  __device__ __forceinline__ uint32_t bin(float d2) const {
    if (lut_shift) {
      const uint32_t u = __float_as_uint(d2);
      const uint32_t e = lut[max((int32_t)(u >> lut_shift) - (int32_t)lut_base, 0)];
      return (e >> 17) + ((u & lut_mask) >= (e & 0x1FFFFu) ? 1u : 0u);
    }
    return bin_index(d2, sE, nb, r0f, inv_dr);
  }

  // one in-range pair (d2 < Emax) of weight w: the RDF bin, or the count below E[0].  The pairs
  // binned are not counted here: the flushes add the rows' sums to the meta array.
  __device__ __forceinline__ void pair_w(float d2, uint32_t w, uint32_t& below) {
    if (!RDF) return;
    if (E0 == 0.f && priv) {  // r0 = 0: every pair (d2 >= 0) is binned (uniform branch)
      atomicAdd(&s_rdfw[bin(d2)], w);
      return;
    }
    const bool in = d2 >= E0;
    const uint32_t b = bin(in ? d2 : E0);
    if (priv)
      atomicAdd(&s_rdfw[b], in ? w : 0u);
    else
      atomicAdd(&s_rdf[b], (unsigned long long)(in ? w : 0u));
    below += in ? 0u : w;
  }
  __device__ __forceinline__ void pair(const QueryArgs& a, float d2, uint32_t& below) { pair_w(d2, 1u, below); }

  // one in-range pair of weight w counted straight into the global histogram (and into binned)
  __device__ __forceinline__ void pair_global(const QueryArgs& a, float d2, uint32_t w, uint64_t& binned,
                                              uint32_t& below) {
    if (!RDF) return;
    if (d2 >= E0) {
      atomicAdd((unsigned long long*)&a.rdf[bin(d2)], (unsigned long long)w);
      binned += w;
    } else {
      below += w;
    }
  }

  // the k-th distance D of one central for the q-th requested k
  __device__ __forceinline__ void kth(const QueryArgs& a, uint32_t q, float D, uint32_t idx) {
    if (a.kth) a.kth[(int64_t)q * a.n + idx] = D;
    uint32_t* sp;
    if (!(D < Emax))
      sp = &s_kmeta[2 * q];
    else if (D < E0)
      sp = &s_kmeta[2 * q + 1];
    else
      sp = &s_knn[q * nb + bin_index(D, sE, nb, r0f, inv_dr)];
    atomicAdd(sp, 1u);
  }

  // one warp adds its private RDF row to the global histogram (and its sum to the pair count)
  // and clears it
  __device__ void flush_warp(const QueryArgs& a) {
    if (!RDF || !priv) return;
    __syncwarp();
    unsigned long long tot = 0;
    for (uint32_t b = threadIdx.x & 31; b < nb; b += 32)
      if (s_rdfw[b]) {
        tot += s_rdfw[b];
        atomicAdd((unsigned long long*)&a.rdf[b], (unsigned long long)s_rdfw[b]);
        s_rdfw[b] = 0;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd((unsigned long long*)&a.meta[PS_META_N_PAIRS], tot);
    __syncwarp();
  }

  // add the shared counters to the global histograms and clear them (whole CTA); the
  // per-warp rows are summed in the CTA first, one global atomic per bin and CTA
  __device__ void flush(const QueryArgs& a) {
    __syncthreads();
    unsigned long long tot = 0;  // pairs binned in this CTA's rows
    if (RDF && priv) {
      uint32_t* rows = reinterpret_cast<uint32_t*>(s_rdf);
      const uint32_t nw = blockDim.x >> 5;
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        unsigned long long sum = 0;
        for (uint32_t w = 0; w < nw; ++w) sum += rows[w * nb + b], rows[w * nb + b] = 0;
        if (sum) atomicAdd((unsigned long long*)&a.rdf[b], sum);
        tot += sum;
      }
    }
    if (RDF && !priv)
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        if (s_rdf[b]) tot += s_rdf[b], atomicAdd((unsigned long long*)&a.rdf[b], s_rdf[b]), s_rdf[b] = 0;
    if (RDF) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd((unsigned long long*)&a.meta[PS_META_N_PAIRS], tot);
    }
    for (uint32_t b = threadIdx.x; b < a.n_k * nb; b += blockDim.x)
      if (s_knn[b]) atomicAdd((unsigned long long*)&a.knn[b], (unsigned long long)s_knn[b]), s_knn[b] = 0;
    for (uint32_t b = threadIdx.x; b < 2 * a.n_k; b += blockDim.x)
      if (s_kmeta[b])
        atomicAdd((unsigned long long*)&a.meta[PS_META_HEAD + b], (unsigned long long)s_kmeta[b]), s_kmeta[b] = 0;
    __syncthreads();
  }
};

// pair counters of the whole CTA (every thread calls it): summed in the warp, then in shared
// memory, one global atomic per counter and CTA
__device__ __forceinline__ void add_pair_counters(const QueryArgs& a, uint64_t binned, uint64_t below) {
  // binned: only the pairs counted straight into the global histogram (the shared rows' pairs
  // are added by the flushes); below: pairs with d2 < E[0]
  __shared__ unsigned long long s_pc[2];
  if (threadIdx.x == 0) s_pc[0] = 0, s_pc[1] = 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    binned += __shfl_xor_sync(0xffffffffu, binned, o);
    below += __shfl_xor_sync(0xffffffffu, below, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    if (binned) atomicAdd(&s_pc[0], (unsigned long long)binned);
    if (below) atomicAdd(&s_pc[1], (unsigned long long)below);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_pc[0]) atomicAdd((unsigned long long*)&a.meta[PS_META_N_PAIRS], s_pc[0]);
    if (s_pc[1]) atomicAdd((unsigned long long*)&a.meta[PS_META_N_BELOW], s_pc[1]);
  }
}

// Rows of the stencil, nearest first: (dy, dz) ordered by dy^2 + dz^2 (the first 9 entries are
// the 3 x 3 rows of the 27-cell stencil, the first 25 the 5 x 5 rows).  Walking the central row
// first lets the k-th distance of every central settle early, so later candidates rarely enter
// the top-k lists.
__constant__ signed char c_row_dy[kMaxRuns] = {0, -1, 1, 0, 0, -1, 1, -1, 1, -2, 2, 0, 0, -2, 2, -2, 2,
                                               -1, 1, -1, 1, -2, 2, -2, 2, 0, 0, -3, 3, -1, 1, -1, 1,
                                               -3, 3, -3, 3, -2, 2, -2, 2, -3, 3, -3, 3, -3, 3, -3, 3};
__constant__ signed char c_row_dz[kMaxRuns] = {0, 0, 0, -1, 1, -1, -1, 1, 1, 0, 0, -2, 2, -1, -1, 1, 1,
                                               -2, -2, 2, 2, -2, -2, 2, 2, -3, 3, 0, 0, -3, -3, 3, 3,
                                               -1, -1, 1, 1, -3, -3, 3, 3, -2, -2, 2, 2, -3, -3, 3, 3};

__device__ __forceinline__ int row_width(const QueryArgs& a, int dy, int dz) {
  const int s = a.stencil;
  return a.row_w[(dz + s) * (2 * s + 1) + dy + s];
}

// x-run of cells cx - w .. cx + w (clipped to the grid) of row (y, z): its records
__device__ __forceinline__ void row_run(const QueryArgs& a, const Geo& ng, uint32_t cx, int y, int z, int w,
                                        uint32_t& src, uint32_t& len) {
  src = 0;
  len = 0;
  if (w < 0 || y < 0 || z < 0 || y >= (int)ng.dims[1] || z >= (int)ng.dims[2]) return;
  const uint32_t xlo = cx >= (uint32_t)w ? cx - w : 0;
  const uint32_t xhi = cx + w < ng.dims[0] ? cx + w : ng.dims[0] - 1;
  const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
  src = a.nstart[row + xlo];
  len = a.nstart[row + xhi + 1] - src;
}

// cell c -> run r of its stencil: the x-contiguous records of cells (cx-w .. cx+w, cy+dy, cz+dz)
__device__ __forceinline__ void cell_run(const QueryArgs& a, const Geo& ng, uint32_t c, uint32_t r, uint32_t& src,
                                         uint32_t& len) {
  const int s = a.stencil, w = 2 * s + 1;
  const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
  src = 0;
  len = 0;
  if ((int)r >= w * w) return;
  const int dy = c_row_dy[r], dz = c_row_dz[r];
  row_run(a, ng, cx, (int)cy + dy, (int)cz + dz, row_width(a, dy, dz), src, len);
}

// Near kNN pass of the query in passes (vertex != 0): the central list is sorted by the grid
// of cells centred on the vertices of the neighbour grid (vg: origin half a cell lower, one more
// cell per axis), so the centrals of item cell c are those nearest to vertex V = c's coordinates,
// and the 2 x 2 x 2 neighbour cells V - 1 .. V along each axis hold every record within half a
// cell of each of them: 4 rows of 2 cells, ~8 cells of candidates instead of the 27 around a
// central's cell.  Run r < 4 of that block:
__device__ __forceinline__ void vertex_run(const QueryArgs& a, const Geo& ng, const Geo& vg, uint32_t c, uint32_t r,
                                           uint32_t& src, uint32_t& len) {
  src = 0;
  len = 0;
  if (r >= 4) return;
  const int vx = (int)(c % vg.dims[0]), vy = (int)((c / vg.dims[0]) % vg.dims[1]), vz = (int)(c / (vg.dims[0] * vg.dims[1]));
  const int y = vy - 1 + (int)(r & 1u), z = vz - 1 + (int)(r >> 1);
  const int xlo = max(vx - 1, 0), xhi = min(vx, (int)ng.dims[0] - 1);
  if (y < 0 || z < 0 || y >= (int)ng.dims[1] || z >= (int)ng.dims[2] || xlo > xhi) return;
  const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
  src = a.nstart[row + xlo];
  len = a.nstart[row + xhi + 1] - src;
}

// The squared reach of central p in vertex cell c: the distance from p to the nearest face of
// its block (cells V - 1 and V along each axis, faces at u = V - 1 and u = V + 1 in the
// neighbour grid's cell coordinate u = (x - origin) * inv_h), less a slack for the float32
// rounding of the cell coordinates of p and of any record (a few ulps of u, below slack cells),
// times the cell edge, shrunk by 2^-12 before and after squaring: every record outside the
// block has d2 above it, so a k-th distance below it is the k-th distance over the whole cloud.
// Capped at E[nb].
__device__ __forceinline__ float vertex_reach(const Geo& ng, const Geo& vg, uint32_t c, const float4& p, float slack,
                                              float h_eff, float Emax) {
  const uint32_t v[3] = {c % vg.dims[0], (c / vg.dims[0]) % vg.dims[1], c / (vg.dims[0] * vg.dims[1])};
  const float pc[3] = {p.x, p.y, p.z};
  float m = INFINITY;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float u = __fmul_rn(__fsub_rn(pc[ax], ng.origin[ax]), ng.inv_h);
    m = fminf(m, fminf(__fsub_rn(u, (float)v[ax] - 1.0f), __fsub_rn((float)v[ax] + 1.0f, u)));
  }
  const float r = __fmul_rn(fmaxf(__fsub_rn(m, slack), 0.0f), h_eff);
  return fminf(__fmul_rn(__fmul_rn(r, r), 1.0f - 1.0f / 4096.0f), Emax);
}

// Lists the centrals (positions in the central list) of the lanes with miss set, warp-aggregated
// (all 32 lanes call it).
__device__ __forceinline__ void list_append(const QueryArgs& a, bool miss, uint32_t pos, uint32_t lane) {
  const uint32_t m = __ballot_sync(0xffffffffu, miss);
  if (!m) return;
  uint32_t at = 0;
  if (lane == 0) at = atomicAdd(&a.cgeo->list_n, (uint32_t)__popc(m));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (miss) a.need[at + __popc(m & ((1u << lane) - 1u))] = pos;
}

__device__ __forceinline__ float4 far_record() { return make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(~0u)); }

// ---------------------------------------------------------------------------
// warp kernel
//   heavy items (cells with >= kHeavy centrals, batches of 4..32 centrals): one
//     to eight lanes per central (item_lanes), the candidates staged 32 at a
//     time in the warp's shared buffer and tested two at a time with packed
//     float32 math;
//   light items (cells with < kHeavy centrals): the warp takes 32 items at a
//     time and gives each of their centrals a thread of its own that walks its
//     own stencil (the records of neighbouring centrals' cells hit in L1).
// ---------------------------------------------------------------------------
constexpr uint32_t kHalf = 16;                 // candidates per staging half-batch
constexpr uint32_t kRowLaneCap = 1u << 25;     // per-central increments of the 32-bit warp row, then global

// VX: the near kNN pass on the vertex-centred central list (a.vertex; kNN only), compiled apart
// so that the other forms carry none of its code
template <int KMAX, bool RDF, bool VX = false>
__global__ void __launch_bounds__(256) k_query_warp(const QueryArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_buf[8][32];
  __shared__ float s_hits[8][32 * kHalf + 32];  // per warp: the in-range hits of one half-batch + a trash row
  __shared__ float s_kq[8][32 * kHalf + 32];    // per warp: kNN insertion queue, [slot][lane] + a spare row
  __shared__ uint32_t s_rsrc[8][kMaxRuns], s_rpre[8][kMaxRuns + 1];
  constexpr int KK = KMAX > 0 ? KMAX : 1;
  Hist<RDF> H;
  H.init(a, smem, 0, true);
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t wcount = 0;  // increments of this warp's private row since its last flush (uniform)
  const Geo ng = *a.ngeo;
  const uint32_t n_hi = a.cgeo->work_n4, n_front = n_hi + a.cgeo->work_n2, n_light = a.cgeo->work_n3;
  const int n_runs = VX ? 4 : (2 * a.stencil + 1) * (2 * a.stencil + 1);
  const float erange = a.emax_near > 0.f ? a.emax_near : H.Emax;  // squared search range of this pass
  // vertex mode: the item cells are those of the vertex-centred grid (a.cgeo); rounding slack of
  // a cell coordinate (cells) and the cell edge for vertex_reach
  const Geo vg = *a.cgeo;
  const float v_slack = (float)max(ng.dims[0], max(ng.dims[1], ng.dims[2])) * 5.0e-7f + 1.0e-6f;
  const float v_heff = __fmul_rn(__fdiv_rn(1.0f, ng.inv_h), 1.0f - 1.0f / 4096.0f);
  uint64_t my_binned = 0;  // pairs counted straight into the global histogram
  uint32_t my_below = 0;   // pairs below E[0]
  float4* buf = s_buf[w];
  float* wlist = s_hits[w];
  float* kq = s_kq[w];
  uint32_t* rsrc = s_rsrc[w];
  uint32_t* rpre = s_rpre[w];

  // ---- items from the front: dense cells, the very heavy ones first ----
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.next_front, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_front) break;
    const uint2 it = item < n_hi ? a.whi[item] : a.witem[item - n_hi];
    const uint32_t c = it.x, first = it.y >> 6, cnt = it.y & 63u;
    const uint32_t c0 = a.cstart[c] + first;
    // run table: sources and prefix counts of the candidate runs
    const uint32_t n_cand = run_table(lane, n_runs, rsrc, rpre, [&](uint32_t r, uint32_t& src, uint32_t& len) {
      if (VX)
        vertex_run(a, ng, vg, c, r, src, len);
      else
        cell_run(a, ng, c, r, src, len);
    });

    // record at virtual candidate position pos (runs concatenated); rr is a run hint, nondecreasing in pos
    auto fetch = [&](uint32_t pos, int& rr) -> float4 {
      if (pos >= n_cand) return far_record();
      while (pos >= rpre[rr + 1]) ++rr;
      return __ldg(a.nrec + rsrc[rr] + (pos - rpre[rr]));
    };

    if (cnt > 3) {
      // 32 candidates per coalesced load, staged as 16 interleaved pairs (xa xb ya yb za zb wa wb)
      // and tested two at a time.  In-range hits go to a warp-wide list (ballot + popc give each
      // hit its slot) binned by all 32 lanes together; kNN candidates below the lane's current
      // k-th distance go to the lane's column of the insertion queue, drained after each half-batch
      // (the sorted insertion then runs with most lanes active instead of once per candidate
      // whenever any lane needs it).
      // L lanes per central (items of dense clusters, a cell's partial last item): lane sub of a
      // central tests the pairs t = sub mod L
      const uint32_t L = item_lanes(cnt);
      const uint32_t lg = L == 8u ? 3u : (L == 4u ? 2u : (L == 2u ? 1u : 0u));
      const uint32_t sub = lane & (L - 1u), ci = lane >> lg;
      const uint32_t n_it = 8u >> lg;  // pair tests per lane per half-batch
      bool valid = ci < cnt;
      if (a.fallback && valid) valid = a.need[c0 + ci] != 0u;
      if (a.fallback && __ballot_sync(0xffffffffu, valid) == 0u) continue;  // no central of this item to redo
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) p = a.crec[c0 + ci];
      const uint32_t pidx = valid ? __float_as_uint(p.w) : ~0u;
      // lanes without a central never hit; vertex mode: each central's own reach
      const float emax = valid ? (VX ? vertex_reach(ng, vg, c, p, v_slack, v_heff, H.Emax) : erange) : -INFINITY;
      const unsigned long long px = f2_pack(p.x, p.x), py = f2_pack(p.y, p.y), pz = f2_pack(p.z, p.z);
      const uint32_t lt = (1u << lane) - 1u;
      float top[KK];
#pragma unroll
      for (int t = 0; t < KK; ++t) top[t] = INFINITY;
      uint32_t within = 0;
      int rr = 0;
      float4 nxt = fetch(lane, rr);
      float* bf = reinterpret_cast<float*>(buf);
      for (uint32_t b = 0; b < n_cand; b += 32) {
        __syncwarp();
        {
          float* d = bf + (lane >> 1) * 8 + (lane & 1);
          d[0] = nxt.x, d[2] = nxt.y, d[4] = nxt.z, d[6] = nxt.w;
        }
        __syncwarp();
        nxt = fetch(b + 32 + lane, rr);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
          uint32_t nh = 0;  // hits in the warp list (uniform)
          uint32_t qn = 0;  // entries in this lane's queue column
          const float thr = top[KK - 1];
          // vertex mode: no in-range count, one bound for the queue (the reach and the k-th distance)
          const float thr_e = fminf(thr, emax);
#pragma unroll 2
          for (uint32_t u = 0; u < n_it; ++u) {
            const uint32_t t = 8 * half + u * L + sub;
            const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(bf)[2 * t];
            const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(bf)[2 * t + 1];
            float d2a, d2b;
            dist2_x2(px, py, pz, xy.x, xy.y, zw.x, d2a, d2b);
            float wa, wb;
            f2_unpack(zw.y, wa, wb);
            if constexpr (VX) {
              const bool qa = d2a < thr_e && __float_as_uint(wa) != pidx;
              const bool qb = d2b < thr_e && __float_as_uint(wb) != pidx;
              kq[qn * 32 + lane] = d2a;
              qn += (uint32_t)qa;
              kq[qn * 32 + lane] = d2b;
              qn += (uint32_t)qb;
              continue;
            }
            const bool ha = d2a < emax && __float_as_uint(wa) != pidx;
            const bool hb = d2b < emax && __float_as_uint(wb) != pidx;
            within += (uint32_t)ha + (uint32_t)hb;
            if (KMAX > 0) {
              // unconditional stores at the queue's next slot (row qn <= 16 of 17), kept only if counted
              const bool qa = ha && d2a < thr, qb = hb && d2b < thr;
              kq[qn * 32 + lane] = d2a;
              qn += (uint32_t)qa;
              kq[qn * 32 + lane] = d2b;
              qn += (uint32_t)qb;
            }
            if (RDF) {
              // every lane stores (no branch): a hit at its compacted slot, a miss in the trash row
              const uint32_t ba = __ballot_sync(0xffffffffu, ha);
              wlist[ha ? nh + __popc(ba & lt) : 32 * kHalf + lane] = d2a;
              nh += __popc(ba);
              const uint32_t bb = __ballot_sync(0xffffffffu, hb);
              wlist[hb ? nh + __popc(bb & lt) : 32 * kHalf + lane] = d2b;
              nh += __popc(bb);
            }
          }
          if (KMAX > 0) {
            const uint32_t m = __reduce_max_sync(0xffffffffu, qn);
            for (uint32_t q = 0; q < m; ++q)
              if (q < qn) topk_insert(top, kq[q * 32 + lane]);
          }
          if (RDF) {
            __syncwarp();
            for (uint32_t h = lane; h < nh; h += 32) H.pair(a, wlist[h], my_below);
            __syncwarp();
            wcount += nh;
            if (wcount >= (1ull << 31)) {
              H.flush_warp(a);
              wcount = 0;
            }
          }
        }
      }
      // merge the partial lists of the L lanes of each central (disjoint candidate subsets); the
      // partner's sorted list is read from the warp's queue buffer in a rolled loop, which keeps
      // the kernel's code small (its speed depends on the instruction cache)
      for (uint32_t o = 1; o < L; o <<= 1) {
        within += __shfl_xor_sync(0xffffffffu, within, o);
        if constexpr (KMAX > 0 && KK * 32 <= 32 * kHalf) {
          __syncwarp();
#pragma unroll
          for (int t = 0; t < KK; ++t) kq[t * 32 + lane] = top[t];
          __syncwarp();
          const float* ot = kq + (lane ^ o);
#pragma unroll 1
          for (int t = 0; t < KK; ++t) {
            const float v = ot[t * 32];
            if (!(v < top[KK - 1])) break;  // the partner's list is sorted
            topk_insert(top, v);
          }
        } else if constexpr (KMAX > 0) {
          float other[KK];
#pragma unroll
          for (int t = 0; t < KK; ++t) other[t] = __shfl_xor_sync(0xffffffffu, top[t], o);
#pragma unroll
          for (int t = 0; t < KK; ++t) {
            if (!(other[t] < top[KK - 1])) break;  // the partner's list is sorted
            topk_insert(top, other[t]);
          }
        }
      }
      bool miss = false;
      if (valid && sub == 0) {
        if (a.nwithin) a.nwithin[pidx] = within;
        if (KMAX > 0) {
          const float kd = topk_get(top, a.k_need - 1);
          const bool found = VX ? kd < emax : (!(a.emax_near > 0.f) || kd < a.emax_near);
          if (VX)
            miss = !found;
          else if (a.emax_near > 0.f)
            a.need[c0 + ci] = found ? 0u : 1u;
          if (found)
            for (uint32_t q = 0; q < a.n_k; ++q) H.kth(a, q, topk_get(top, a.ks[q] - 1), pidx);
        }
      }
      if (VX) list_append(a, miss, c0 + ci, lane);
    } else {
      // few centrals, many candidates: the lanes split the candidates of each central and
      // merge their sorted lists by shuffles
      for (uint32_t ci = 0; ci < cnt; ++ci) {
        if (a.fallback && a.need[c0 + ci] == 0u) continue;  // warp-uniform
        const float4 p = a.crec[c0 + ci];
        const uint32_t pidx = __float_as_uint(p.w);
        const float er = VX ? vertex_reach(ng, vg, c, p, v_slack, v_heff, H.Emax) : erange;
        float top[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) top[t] = INFINITY;
        uint32_t within = 0;
        int rr = 0;
        for (uint32_t b = 0; b < n_cand; b += 32) {
          const float4 q = fetch(b + lane, rr);
          const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
          if (d2 < er && __float_as_uint(q.w) != pidx) {
            ++within;
            H.pair(a, d2, my_below);
            if (KMAX > 0) topk_insert(top, d2);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) within += __shfl_xor_sync(0xffffffffu, within, o);
        if (lane == 0 && a.nwithin) a.nwithin[pidx] = within;
        wcount += within;
        if (wcount >= (1ull << 31)) {
          H.flush_warp(a);
          wcount = 0;
        }
        if (KMAX > 0) {
          // merge the 32 sorted lane lists: pop the warp minimum k_need times (ranks kept in kq)
          float m = INFINITY;
          for (uint32_t rank = 0; rank < a.k_need; ++rank) {
            m = top[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            const uint32_t bal = __ballot_sync(0xffffffffu, top[0] == m);
            if (lane == (uint32_t)(__ffs(bal) - 1)) {
#pragma unroll
              for (int t = 0; t < KK - 1; ++t) top[t] = top[t + 1];
              top[KK - 1] = INFINITY;
            }
            if (lane == 0) kq[rank] = m;
          }
          __syncwarp();
          if (lane == 0) {
            const bool found = VX ? m < er : (!(a.emax_near > 0.f) || m < a.emax_near);
            if (VX) {
              if (!found) a.need[atomicAdd(&a.cgeo->list_n, 1u)] = c0 + ci;
            } else if (a.emax_near > 0.f) {
              a.need[c0 + ci] = found ? 0u : 1u;
            }
            if (found)
              for (uint32_t q = 0; q < a.n_k; ++q) H.kth(a, q, kq[a.ks[q] - 1], pidx);
          }
          __syncwarp();
        }
      }
    }
  }

  // ---- items from the back: sparse cells, one thread per central ----
  // central record and cell of the taken items' centrals (<= 32 * 15, kHeavy - 1 per item)
  uint32_t* cl_rec = reinterpret_cast<uint32_t*>(s_hits[w]);
  uint32_t* cl_cell = reinterpret_cast<uint32_t*>(s_kq[w]);
  const int st = a.stencil;
  // items per take: enough that every warp of the grid gets work when the list is short
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t take = min(32u, max(1u, (n_light + n_warps - 1) / n_warps));
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(a.next_light, take);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_light) break;
    uint32_t c = 0, f = 0, cnt = 0;
    if (lane < take && base + lane < n_light) {
      const uint2 it = a.witem[a.work_cap - 1 - (base + lane)];
      c = it.x;
      f = a.cstart[c] + (it.y >> 6);
      cnt = it.y & 63u;
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    __syncwarp();
    for (uint32_t q = 0; q < cnt; ++q) cl_rec[inc - cnt + q] = f + q, cl_cell[inc - cnt + q] = c;
    __syncwarp();
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
      bool valid = r0 + lane < total;
      if (a.fallback && valid) valid = a.need[cl_rec[r0 + lane]] != 0u;
      uint32_t rowc = 0;  // increments of the warp row by this lane
      if (valid) {
        const uint32_t ce = cl_cell[r0 + lane];
        const float4 p = __ldg(a.crec + cl_rec[r0 + lane]);
        const uint32_t pidx = __float_as_uint(p.w);
        const uint32_t cx = ce % ng.dims[0], cy = (ce / ng.dims[0]) % ng.dims[1], cz = ce / (ng.dims[0] * ng.dims[1]);
        float top[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) top[t] = INFINITY;
        uint32_t within = 0;
        for (int dz = -st; dz <= st; ++dz)
          for (int dy = -st; dy <= st; ++dy) {
            uint32_t j0 = 0, nj = 0;
            row_run(a, ng, cx, (int)cy + dy, (int)cz + dz, row_width(a, dy, dz), j0, nj);
            const uint32_t j1 = j0 + nj;
            for (uint32_t j = j0; j < j1; ++j) {
              const float4 q = __ldg(a.nrec + j);
              const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
              if (d2 < erange && __float_as_uint(q.w) != pidx) {
                ++within;
                if (RDF) {
                  if (within <= kRowLaneCap)
                    H.pair(a, d2, my_below);
                  else
                    H.pair_global(a, d2, 1u, my_binned, my_below);
                }
                if (KMAX > 0 && d2 < top[KK - 1]) topk_insert(top, d2);
              }
            }
          }
        rowc = within < kRowLaneCap ? within : kRowLaneCap;
        if (a.nwithin) a.nwithin[pidx] = within;
        if (KMAX > 0) {
          const bool found = !(a.emax_near > 0.f) || topk_get(top, a.k_need - 1) < a.emax_near;
          if (a.emax_near > 0.f) a.need[cl_rec[r0 + lane]] = found ? 0u : 1u;
          if (found)
            for (uint32_t q = 0; q < a.n_k; ++q) H.kth(a, q, topk_get(top, a.ks[q] - 1), pidx);
        }
      }
      if (RDF) {
        // a round adds at most 32 * 2^25 = 2^30 to the row: flushed at 2^31, it never wraps
        wcount += __reduce_add_sync(0xffffffffu, rowc);
        if (wcount >= (1ull << 31)) {
          H.flush_warp(a);
          wcount = 0;
        }
      }
    }
    __syncwarp();  // cl is rewritten next
  }
  H.flush(a);
  add_pair_counters(a, my_binned, my_below);
}

// ---------------------------------------------------------------------------
// CTA kernel: one CTA per dense cell, runs staged in shared memory by bulk copies
// ---------------------------------------------------------------------------
template <int KMAX, bool RDF>
__global__ void __launch_bounds__(256) k_query_cta(const QueryArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t s_item;
  __shared__ uint32_t s_run_src[kMaxRuns], s_run_len[kMaxRuns];
  __shared__ int s_timeout;
  constexpr int KK = KMAX > 0 ? KMAX : 1;

  Hist<RDF> H;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_timeout = 0;
  }
  H.init(a, smem, a.stage_cap);
  float4* s_cand =
      reinterpret_cast<float4*>(smem + smem_layout(a.n_bins, a.n_k, RDF, a.stage_cap, false, a.lut_n).off_stage);
  const uint32_t tid = threadIdx.x;
  const Geo ng = *a.ngeo;
  const uint32_t work_n = a.cgeo->work_n;
  const uint32_t n_runs = (2 * a.stencil + 1) * (2 * a.stencil + 1);
  uint32_t phase = 0, stuck_phase = 0;
  uint64_t my_binned = 0;
  uint32_t my_below = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.cgeo->work_next, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= work_n || s_timeout) break;
    const uint32_t c = a.cwork[item];
    const uint32_t c0 = a.cstart[c], n_c = a.cstart[c + 1] - c0;
    if (tid < n_runs) cell_run(a, ng, c, tid, s_run_src[tid], s_run_len[tid]);
    __syncthreads();

    for (uint32_t cb = 0; cb < n_c; cb += blockDim.x) {
      const uint32_t ci = cb + tid;
      const bool valid = ci < n_c;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) p = a.crec[c0 + ci];
      const uint32_t pidx = __float_as_uint(p.w);
      float top[KK];
#pragma unroll
      for (int t = 0; t < KK; ++t) top[t] = INFINITY;
      uint32_t within = 0;

      // walk the runs in chunks of at most stage_cap records (padded to a multiple of 8 with far records)
      uint32_t r = 0, ro = 0;
      while (r < n_runs) {
        uint32_t chunk = 0;
        uint32_t rr = r, rro = ro;
        while (rr < n_runs && chunk < a.stage_cap) {
          const uint32_t len = s_run_len[rr];
          const uint32_t take = min(len - rro, a.stage_cap - chunk);
          chunk += take;
          rro += take;
          if (rro >= len) ++rr, rro = 0;
        }
        if (chunk == 0) break;
        const uint32_t padded = (chunk + 7u) & ~7u;
        if (tid == 0) {
          for (uint32_t t = chunk; t < padded; ++t) s_cand[t] = far_record();
          mbar_arrive_expect_tx(&bar, chunk * 16u);
          uint32_t dst = 0, q = r, qo = ro;
          while (q < n_runs && dst < chunk) {
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
        const uint32_t this_phase = phase;
        phase ^= 1u;

        if (valid) {
          for (uint32_t t0 = 0; t0 < padded; t0 += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float4 q = s_cand[t0 + u];
              const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
              if (d2 < H.Emax && __float_as_uint(q.w) != pidx) {
                ++within;
                H.pair(a, d2, my_below);
                if (KMAX > 0) topk_insert(top, d2);
              }
            }
          }
        }
        __syncthreads();  // the chunk buffer is reused next
        if (s_timeout) {  // uniform after the barrier: issue no more copies
          stuck_phase = this_phase;
          break;
        }
      }
      if (s_timeout) break;
      if (valid) {
        if (a.nwithin) a.nwithin[pidx] = within;
        if (KMAX > 0)
          for (uint32_t q = 0; q < a.n_k; ++q) H.kth(a, q, topk_get(top, a.ks[q] - 1), pidx);
      }
    }
    __syncthreads();  // s_item and the run table are rewritten next
  }
  if (s_timeout) {
    // the copies of the phase that timed out may still be in flight into this CTA's shared
    // memory: wait for them once more (bounded) before the CTA exits
    if (tid == 0) mbar_wait_bounded(&bar, stuck_phase, kWaitLimitNs);
    __syncthreads();
  }
  H.flush(a);
  add_pair_counters(a, my_binned, my_below);
  if (tid == 0 && s_timeout) atomicCAS((int*)&a.cgeo->status, 0, (int)PS_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// symmetric RDF pass: every unordered pair of neighbour records once
//
// The RDF counts ordered pairs (i central, j neighbour, j != i).  When the centrals are
// neighbour records, an unordered pair {i, j} contributes c_i + c_j (c = 1 for a central
// record), and d2_ij == d2_ji bit for bit (x_j - x_i == -(x_i - x_j) in IEEE arithmetic), so
// each pair is tested once, from the lower of its two cells: the half of the stencil with
// (dz > 0) or (dz == 0 and dy > 0) or (dz == dy == 0 and dx > 0), plus the pairs i < j inside
// the cell.  A warp takes 32 cells at a time, and for each non-empty cell tests the half
// stencil's records (the lanes, 32 per load) against the cell's records (staged in shared
// memory, read by all lanes at once, two at a time with packed float32 math); the hits (d2,
// weight) are compacted into a warp list and binned into the warp's 32-bit shared row by all
// lanes.  The flags come from the central prefix pfx over the records (c_j = pfx[j+1] - pfx[j]).
// ---------------------------------------------------------------------------

// half-stencil run r of cell c: the x-runs of the rows with dz > 0 (all dy) and of the rows
// dz == 0, dy > 0 (each over its width, see row_width); the row dz == dy == 0 from cx + 1 on.
// (2s+1)s + s + 1 runs.
__device__ __forceinline__ void sym_run(const QueryArgs& a, const Geo& ng, uint32_t c, uint32_t r, uint32_t& src,
                                        uint32_t& len) {
  const int s = a.stencil, W = 2 * s + 1;
  const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
  src = 0;
  len = 0;
  int dy, dz;
  if ((int)r < W * s) {
    dz = 1 + (int)r / W;
    dy = (int)r % W - s;
  } else if ((int)r < W * s + s) {
    dz = 0;
    dy = 1 + ((int)r - W * s);
  } else if ((int)r == W * s + s) {
    // own row, the cells after c: cx + 1 .. cx + s
    const uint32_t xhi = cx + s < ng.dims[0] ? cx + s : ng.dims[0] - 1;
    if (cx + 1 <= xhi) {
      const uint32_t row = (cz * ng.dims[1] + cy) * ng.dims[0];
      src = a.nstart[row + cx + 1];
      len = a.nstart[row + xhi + 1] - src;
    }
    return;
  } else {
    return;
  }
  row_run(a, ng, cx, (int)cy + dy, (int)cz + dz, row_width(a, dy, dz), src, len);
}

constexpr uint32_t kSymGroup = 64;  // records of a cell staged at a time by the symmetric pass

__global__ void __launch_bounds__(256, 4) k_rdf_sym(const QueryArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_grp[8][kSymGroup];          // per warp: the cell's records as interleaved pairs
  __shared__ uint32_t s_hits[8][32 * kHalf + 32];  // per warp: the hits of 8 record pairs + a trash row: the
                                                  // bits of d2, the sign bit set for weight 2
  __shared__ uint32_t s_rsrc[8][kMaxRuns], s_rpre[8][kMaxRuns + 1];
  Hist<true> H;
  H.init(a, smem, 0, true);
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t wcount = 0;  // increments of this warp's private row since its last flush (uniform)
  const Geo ng = *a.ngeo;
  const uint32_t n_cells = ng.n_cells;
  const int s = a.stencil, n_runs = (2 * s + 1) * s + s + 1;
  uint64_t my_binned = 0;
  uint32_t my_below = 0;
  float* gf = reinterpret_cast<float*>(s_grp[w]);
  uint32_t* wlist = s_hits[w];
  uint32_t* rsrc = s_rsrc[w];
  uint32_t* rpre = s_rpre[w];
  const float E_max = H.Emax;

  // cells per take: a share of the cells left (at most 32, at least 1), so that the warps finish
  // together -- a take of 32 cells is a large part of a warp's work on a small grid
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  for (;;) {
    uint32_t base = 0, take = 0;
    if (lane == 0) {
      const uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&a.cgeo->sym_next);
      const uint32_t left = cur < n_cells ? n_cells - cur : 0u;
      take = min(32u, max(1u, left / (8 * n_warps)));
      base = atomicAdd(&a.cgeo->sym_next, take);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    take = __shfl_sync(0xffffffffu, take, 0);
    if (base >= n_cells) break;
    uint32_t s0 = 0, s1 = 0;
    if (lane < take && base + lane < n_cells) s0 = a.nstart[base + lane], s1 = a.nstart[base + lane + 1];
    uint32_t todo = __ballot_sync(0xffffffffu, s1 > s0);
    while (todo) {
      const int src_lane = __ffs(todo) - 1;
      todo &= todo - 1u;
      const uint32_t c = base + (uint32_t)src_lane;
      const uint32_t a0 = __shfl_sync(0xffffffffu, s0, src_lane), a1 = __shfl_sync(0xffffffffu, s1, src_lane);
      // run table of the half stencil
      const uint32_t n_cand = run_table(lane, n_runs, rsrc, rpre,
                                        [&](uint32_t r, uint32_t& src, uint32_t& len) { sym_run(a, ng, c, r, src, len); });

      // pairs inside the cell: record i (a lane) with j in (i, a1), each lane on its own (a small
      // share of the pairs)
      for (uint32_t i0 = a0; i0 < a1; i0 += 32) {
        const uint32_t i = i0 + lane;
        uint32_t inc = 0;
        if (i < a1) {
          const float4 p = __ldg(a.nrec + i);
          const uint32_t ci = __ldg(a.pfx + i + 1) - __ldg(a.pfx + i);
          const bool big = a1 - a0 > (1u << 20);  // per-lane increments stay far below the row's 2^32
          for (uint32_t j = i + 1; j < a1; ++j) {
            const float4 q = __ldg(a.nrec + j);
            const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
            const uint32_t wt = ci + (__ldg(a.pfx + j + 1) - __ldg(a.pfx + j));
            if (d2 < E_max && wt) {
              if (big) {
                H.pair_global(a, d2, wt, my_binned, my_below);
              } else {
                H.pair_w(d2, wt, my_below);
                inc += wt;
              }
            }
          }
        }
        wcount += __reduce_add_sync(0xffffffffu, inc);
        if (wcount >= (1ull << 31)) {
          H.flush_warp(a);
          wcount = 0;
        }
      }
      if (n_cand == 0) continue;

      // the half stencil: the candidates are the lanes (32 per coalesced load, each in registers),
      // the cell's records are staged in shared memory (up to kSymGroup at a time, as interleaved
      // pairs xa xb ya yb za zb ea eb) and read by every lane at once, two per packed test; a
      // record's e (and a candidate's) is E[nb] for a central and -1 otherwise, the range of a
      // pair max(e_rec, e_cand), weight 2 (sign bit) when both are central.  The lanes stay busy
      // whatever the cell's record count.
      for (uint32_t g0 = a0; g0 < a1; g0 += kSymGroup) {
        const uint32_t m = min(kSymGroup, a1 - g0), n_pr = (m + 1) >> 1;
        __syncwarp();
#pragma unroll
        for (uint32_t h = 0; h < kSymGroup; h += 32) {
          const uint32_t r = h + lane;
          if (r < 2 * n_pr) {
            float4 q = make_float4(INFINITY, INFINITY, INFINITY, -1.f);  // the pad of an odd group never hits
            if (r < m) {
              q = __ldg(a.nrec + g0 + r);
              q.w = __ldg(a.pfx + g0 + r + 1) > __ldg(a.pfx + g0 + r) ? E_max : -1.f;
            }
            float* d = gf + (r >> 1) * 8 + (r & 1);
            d[0] = q.x, d[2] = q.y, d[4] = q.z, d[6] = q.w;
          }
        }
        __syncwarp();
        int rr = 0;
        auto fetch = [&](uint32_t pos) -> float4 {
          if (pos >= n_cand) return make_float4(INFINITY, INFINITY, INFINITY, -1.f);
          while (pos >= rpre[rr + 1]) ++rr;
          const uint32_t j = rsrc[rr] + (pos - rpre[rr]);
          float4 q = __ldg(a.nrec + j);
          q.w = __ldg(a.pfx + j + 1) > __ldg(a.pfx + j) ? E_max : -1.f;
          return q;
        };
        float4 nxt = fetch(lane);
        for (uint32_t b = 0; b < n_cand; b += 32) {
          const float4 q = nxt;
          nxt = fetch(b + 32 + lane);
          const unsigned long long qx = f2_pack(q.x, q.x), qy = f2_pack(q.y, q.y), qz = f2_pack(q.z, q.z);
          const float eq = q.w;
          const uint32_t w2q = eq > 0.f ? 0x80000000u : 0u;
          for (uint32_t k0 = 0; k0 < n_pr; k0 += 8) {
            const uint32_t k1 = min(n_pr, k0 + 8);
            uint32_t nh = 0;  // hits in the warp list (uniform)
#pragma unroll 4
            for (uint32_t k = k0; k < k1; ++k) {
              const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(gf)[2 * k];
              const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(gf)[2 * k + 1];
              float d2a, d2b;
              dist2_x2(xy.x, xy.y, zw.x, qx, qy, qz, d2a, d2b);
              float ea, eb;
              f2_unpack(zw.y, ea, eb);
              const bool ha = d2a < fmaxf(eq, ea);
              const bool hb = d2b < fmaxf(eq, eb);
              const uint32_t va = __float_as_uint(d2a) | (~__float_as_uint(ea) & w2q);
              const uint32_t vb = __float_as_uint(d2b) | (~__float_as_uint(eb) & w2q);
              // every lane stores (no branch): a hit at its compacted slot, a miss in the trash row
              const uint32_t ba = __ballot_sync(0xffffffffu, ha);
              wlist[ha ? nh + __popc(ba & lt) : 32 * kHalf + lane] = va;
              nh += __popc(ba);
              const uint32_t bb = __ballot_sync(0xffffffffu, hb);
              wlist[hb ? nh + __popc(bb & lt) : 32 * kHalf + lane] = vb;
              nh += __popc(bb);
            }
            __syncwarp();
            for (uint32_t h = lane; h < nh; h += 32) {
              const uint32_t v = wlist[h];
              H.pair_w(__uint_as_float(v & 0x7FFFFFFFu), 1u + (v >> 31), my_below);
            }
            __syncwarp();
            wcount += 2ull * nh;
            if (wcount >= (1ull << 31)) {
              H.flush_warp(a);
              wcount = 0;
            }
          }
        }
      }
    }
  }
  H.flush(a);
  add_pair_counters(a, my_binned, my_below);
}

// ---------------------------------------------------------------------------
// full-radius kNN of the centrals the near pass could not settle
// ---------------------------------------------------------------------------
// Full-radius kNN of the centrals listed by the near pass: one lane per listed central, in two
// tiers: (A) the 27 cells around its cell (every record within one cell of it; the central's
// reach is its distance to the faces of that block, less the rounding slack), then, for the
// warps with a central whose k-th distance is not within that reach, (B) the rest of its stencil
// (the outer cells of the 9 inner rows and the outer rows).  Each tier walks its rows (nearest
// first) with the k_need smallest d2 below E[nb] kept through the per-lane queue; fewer than k of
// them: not found (INF).
template <int KMAX>
__global__ void __launch_bounds__(256) k_knn_list(const QueryArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_kq[8][17 * 32];
  Hist<false> H{};
  H.init(a, smem, 0, true);
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* kq = s_kq[w];
  const Geo ng = *a.ngeo;
  const float Emax = H.Emax;
  const uint32_t n_list = a.cgeo->list_n;
  const int s = a.stencil, n_rows = (2 * s + 1) * (2 * s + 1);
  const float slack = (float)max(ng.dims[0], max(ng.dims[1], ng.dims[2])) * 5.0e-7f + 1.0e-6f;
  const float h_eff = __fmul_rn(__fdiv_rn(1.0f, ng.inv_h), 1.0f - 1.0f / 4096.0f);
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t base = (blockIdx.x * (blockDim.x >> 5) + w) * 32u; base < n_list; base += n_warps * 32u) {
    const bool valid = base + lane < n_list;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    int cc[3] = {0, 0, 0};
    float reach = -1.0f;
    if (valid) {
      p = a.crec[a.need[base + lane]];
      const float pc[3] = {p.x, p.y, p.z};
      float m = INFINITY;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const float u = __fmul_rn(__fsub_rn(pc[ax], ng.origin[ax]), ng.inv_h);
        int c = __float2int_rd(u);
        c = c < 0 ? 0 : (c >= (int)ng.dims[ax] ? (int)ng.dims[ax] - 1 : c);
        cc[ax] = c;
        m = fminf(m, fminf(__fsub_rn(u, (float)c - 1.0f), __fsub_rn((float)c + 2.0f, u)));
      }
      const float r = __fmul_rn(fmaxf(__fsub_rn(m, slack), 0.0f), h_eff);
      reach = fminf(__fmul_rn(__fmul_rn(r, r), 1.0f - 1.0f / 4096.0f), Emax);
    }
    const uint32_t pidx = valid ? __float_as_uint(p.w) : ~0u;
    float top[KMAX];
#pragma unroll
    for (int t = 0; t < KMAX; ++t) top[t] = INFINITY;
    // one x-run per lane: the records of cells xlo..xhi of row (y, z), for the lanes in `act`
    auto walk = [&](bool act, int y, int z, int xlo, int xhi) {
      uint32_t src = 0, len = 0;
      xlo = max(xlo, 0), xhi = min(xhi, (int)ng.dims[0] - 1);
      if (act && xlo <= xhi && y >= 0 && z >= 0 && y < (int)ng.dims[1] && z < (int)ng.dims[2]) {
        const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
        src = a.nstart[row + xlo];
        len = a.nstart[row + xhi + 1] - src;
      }
      const uint32_t n_max = __reduce_max_sync(0xffffffffu, len);
      for (uint32_t t0 = 0; t0 < n_max; t0 += 16) {
        const float thr = fminf(top[KMAX - 1], Emax);  // in range only: fewer than k leaves INF
        uint32_t qn = 0;
#pragma unroll 4
        for (uint32_t u = 0; u < 16; ++u) {
          const uint32_t t = t0 + u;
          float4 q = far_record();
          if (t < len) q = __ldg(a.nrec + src + t);
          const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
          kq[qn * 32 + lane] = d2;
          qn += (d2 < thr && __float_as_uint(q.w) != pidx) ? 1u : 0u;
        }
        const uint32_t m = __reduce_max_sync(0xffffffffu, qn);
        for (uint32_t q = 0; q < m; ++q)
          if (q < qn) topk_insert(top, kq[q * 32 + lane]);
        __syncwarp();
      }
    };
    // tier A: the 9 inner rows over cx - 1 .. cx + 1 (the first 9 rows of the nearest-first order)
    for (int r = 0; r < 9; ++r)
      walk(valid, cc[1] + c_row_dy[r], cc[2] + c_row_dz[r], cc[0] - 1, cc[0] + 1);
    const bool more = valid && !(topk_get(top, a.k_need - 1) < reach);
    if (__ballot_sync(0xffffffffu, more)) {
      // tier B: the outer cells of the inner rows, then the outer rows, each within its width
      for (int r = 0; r < 9; ++r) {
        const int dy = c_row_dy[r], dz = c_row_dz[r], wd = valid ? row_width(a, dy, dz) : -1;
        walk(more && wd >= 2, cc[1] + dy, cc[2] + dz, cc[0] - wd, cc[0] - 2);
        walk(more && wd >= 2, cc[1] + dy, cc[2] + dz, cc[0] + 2, cc[0] + wd);
      }
      for (int r = 9; r < n_rows; ++r) {
        const int dy = c_row_dy[r], dz = c_row_dz[r], wd = valid ? row_width(a, dy, dz) : -1;
        walk(more && wd >= 0, cc[1] + dy, cc[2] + dz, cc[0] - wd, cc[0] + wd);
      }
    }
    if (valid)
      for (uint32_t q = 0; q < a.n_k; ++q) H.kth(a, q, topk_get(top, a.ks[q] - 1), pidx);
  }
  H.flush(a);
}

template <int KMAX>
static int launch_knn_list(const ps_grid* g, const QueryArgs& qa, uint32_t smem, cudaStream_t s) {
  auto k = k_knn_list<KMAX>;
  int per_sm = 0;
  PS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
  if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "full-radius kNN kernel does not fit on an SM");
  PS_LAUNCH(PS_KID_KNN_FULL, s, PS_CUDA(launch_pdl(k, g->num_sms * per_sm, 256, smem, s, qa)));
  return PS_OK;
}

static int dispatch_knn_list(const ps_grid* g, const QueryArgs& qa, uint32_t smem, cudaStream_t s) {
  const uint32_t k = qa.k_need;
  if (k <= 1) return launch_knn_list<1>(g, qa, smem, s);
  if (k <= 2) return launch_knn_list<2>(g, qa, smem, s);
  if (k <= 4) return launch_knn_list<4>(g, qa, smem, s);
  if (k <= 8) return launch_knn_list<8>(g, qa, smem, s);
  if (k <= 10) return launch_knn_list<10>(g, qa, smem, s);
  if (k <= 12) return launch_knn_list<12>(g, qa, smem, s);
  if (k <= 16) return launch_knn_list<16>(g, qa, smem, s);
  return launch_knn_list<32>(g, qa, smem, s);
}

// Writes n_central and the device status into the meta array.
__global__ void k_query_epilogue(const Geo* __restrict__ ngeo, const Geo* __restrict__ cgeo, uint64_t* meta) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) {
    meta[PS_META_N_CENTRAL] = cgeo->n_sel;
    int st = cgeo->status;
    if (st == 0) st = ngeo->status;
    meta[PS_META_STATUS] = (uint64_t)(uint32_t)st;
  }
}

template <int KMAX, bool RDF>
static int launch_query(const ps_grid* g, const QueryArgs& qa, uint32_t smem_cta, uint32_t smem_warp, cudaStream_t s) {
  const uint32_t kid = qa.fallback ? PS_KID_KNN_FULL : PS_KID_QUERY;
  auto kw = (!RDF && qa.vertex) ? k_query_warp<KMAX, RDF, !RDF> : k_query_warp<KMAX, RDF>;
  PS_CUDA(cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_warp));
  int per_sm_w = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_w, kw, 256, smem_warp));
  if (per_sm_w < 1) return fail(PS_ERR_UNSUPPORTED, "query kernel does not fit on an SM");
  if (g->dense_min != 0xFFFFFFFFu) {
    auto kc = k_query_cta<KMAX, RDF>;
    PS_CUDA(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cta));
    int per_sm_c = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, kc, 256, smem_cta));
    if (per_sm_c < 1) return fail(PS_ERR_UNSUPPORTED, "query kernel does not fit on an SM");
    PS_LAUNCH(kid, s, PS_CUDA(launch_pdl(kc, g->num_sms * per_sm_c, 256, smem_cta, s, qa)));
  }
  PS_LAUNCH(kid, s, PS_CUDA(launch_pdl(kw, g->num_sms * per_sm_w, 256, smem_warp, s, qa)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

template <bool RDF>
static int dispatch_k(const ps_grid* g, const QueryArgs& qa, uint32_t sc, uint32_t sw, cudaStream_t s) {
  const uint32_t k = qa.k_need;
  if (k == 0) return RDF ? launch_query<0, RDF>(g, qa, sc, sw, s) : PS_OK;
  if (k <= 1) return launch_query<1, RDF>(g, qa, sc, sw, s);
  if (k <= 2) return launch_query<2, RDF>(g, qa, sc, sw, s);
  if (k <= 4) return launch_query<4, RDF>(g, qa, sc, sw, s);
  if (k <= 8) return launch_query<8, RDF>(g, qa, sc, sw, s);
  if (k <= 10) return launch_query<10, RDF>(g, qa, sc, sw, s);
  if (k <= 12) return launch_query<12, RDF>(g, qa, sc, sw, s);
  if (k <= 16) return launch_query<16, RDF>(g, qa, sc, sw, s);
  return launch_query<32, RDF>(g, qa, sc, sw, s);
}

// Parameters of the bin lookup table: a bit shift S <= 16 at which the interior edges
// E[1..nb-1] fall in strictly increasing cells of the float32 bit pattern (bits >> S), so that a
// cell holds at most one edge, whose low S bits its entry carries; the table covers the cells from
// the one below E[1]'s to E[nb]'s.  The largest such S gives the smallest table.  None when the
// table would exceed kLutMax entries, two edges coincide or nb >= 2^15.
static void choose_lut(ps_bins bins, QueryArgs& qa) {
  qa.lut_shift = qa.lut_base = qa.lut_n = 0;
  const uint32_t nb = bins.n_bins;
  if (nb < 2 || nb >= (1u << 15)) return;
  std::vector<uint32_t> Eb(nb + 1);
  for (uint32_t b = 0; b <= nb; ++b) {
    const double e = bins.r0 + (double)b * bins.dr;
    const float f = (float)(e * e);
    memcpy(&Eb[b], &f, 4);
  }
  for (int S = 16; S >= 1; --S) {
    bool ok = (Eb[1] >> S) >= 1;
    for (uint32_t b = 2; b < nb && ok; ++b) ok = (Eb[b] >> S) > (Eb[b - 1] >> S);
    if (!ok) continue;
    const uint32_t base = (Eb[1] >> S) - 1, n = (Eb[nb] >> S) - base + 1;
    if (n <= kLutMax) {
      qa.lut_shift = (uint32_t)S;
      qa.lut_base = base;
      qa.lut_n = n;
    }
    return;
  }
}

// Row widths of a stencil of s cells for cells of edge h >= r_cut * cs * (1 + 2^-10) (plus the
// grid's rounding margin extent * 2^-20, which covers the float32 rounding of the cell index).
// Two points whose cells are |d| >= 2 apart along an axis are more than (|d| - 1) r_cut cs apart
// along it, so cell offset (dx, dy, dz) can hold a pair within r_cut only if
// sum_i max(0, |d_i| - 1)^2 (cs (1 + 2^-10))^2 < 1; the test keeps a further 2^-20 margin.
// Stencils of three cells (cs < 1/2) lose the 4 far corner cells of each octant; two-cell stencils
// lose corners or rows only for cs above ~0.58.
static void row_widths(int s, double cs, int8_t* w) {
  const int W = 2 * s + 1;
  const double f = cs * (1.0 + 1.0 / 1024.0), lim = (1.0 + 1.0 / 1048576.0) * (1.0 + 1.0 / 1048576.0);
  auto m2 = [](int d) { const int m = d < 0 ? -d - 1 : d - 1; return m > 0 ? (double)(m * m) : 0.0; };
  for (int dz = -s; dz <= s; ++dz)
    for (int dy = -s; dy <= s; ++dy) {
      int width = -1;
      for (int dx = 0; dx <= s; ++dx)
        if ((m2(dx) + m2(dy) + m2(dz)) * f * f < lim) width = dx;
      w[(dz + s) * W + dy + s] = (int8_t)width;
    }
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
  qa.witem = g->ctr.witem;
  qa.whi = g->nbr_witem;
  qa.work_cap = g->item_cap;
  qa.cgeo = g->ctr.geo;
  qa.stencil = g->stencil;
  row_widths(g->stencil, g->cell_scale, qa.row_w);
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
  qa.next_front = &g->ctr.geo->work_next2;
  qa.next_light = &g->ctr.geo->work_next3;
  choose_lut(bins, qa);

  const bool rdf = d_rdf != nullptr;
  ZeroOut z;  // the outputs are zeroed by the central-list reset kernel
  z.p[0] = d_meta;
  z.n[0] = PS_META_LEN(n_k);
  if (rdf) z.p[1] = d_rdf, z.n[1] = bins.n_bins;
  if (n_k) z.p[2] = d_knn, z.n[2] = n_k * bins.n_bins;

  bool subset = !g->pack_type;
  for (int w = 0; w < 4; ++w) subset = subset && (ctr_mask[w] & ~g->nbr_mask[w]) == 0;
  // the query in passes, and its near kNN pass on the vertex-centred central list (two-cell
  // stencils; the ranks of that counting sort take one word per central of the cell arrays)
  const bool split = g->split && subset && rdf && d_nwithin == nullptr && g->stencil >= 2 && g->dense_min == 0xFFFFFFFFu;
  const bool vertex = split && n_k > 0 && g->stencil == 2 && (uint64_t)g->n <= (uint64_t)g->cell_cap;
  int rc = build_central_list(g, dsrf, ctr_mask, dsrf_min, s, z, true, vertex);
  if (rc) return rc;

  // staging budget of the CTA kernel: two CTAs per SM
  int dev_smem = 0;
  PS_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  const SmemLayout base = smem_layout(bins.n_bins, n_k, rdf, 0, false, qa.lut_n);
  const uint32_t budget = (uint32_t)dev_smem / 2 - 2048;
  if (base.total + 16 * 1024 > (uint32_t)dev_smem - 1024)
    return fail(PS_ERR_UNSUPPORTED, "too many bins x k values for shared memory");
  uint32_t stage_bytes = budget > base.total + 16 * 1024 ? budget - base.total : 16 * 1024;
  qa.stage_cap = (stage_bytes / 16) & ~7u;
  const uint32_t smem_cta = smem_layout(bins.n_bins, n_k, rdf, qa.stage_cap, false, qa.lut_n).total;
  const uint32_t smem_warp = smem_layout(bins.n_bins, n_k, rdf, 0, true, qa.lut_n).total;
  if (split) {
    // the query in passes: (1) kNN near each central, centrals with fewer than k_need
    // neighbours there set apart; (2) their full-radius kNN; (3) the RDF over unordered pairs
    if (n_k > 0) {
      QueryArgs qn = qa;
      qn.need = g->sel;  // free between a build and the next one (the counting sort's index list)
      const uint32_t smem_knn = smem_layout(bins.n_bins, n_k, false, 0, true).total;
      if (vertex) {
        // the 2 x 2 x 2 cells around each central's nearest vertex, each central within its own
        // reach (k_query_warp, vertex mode); the others listed for k_knn_list
        qn.vertex = 1;
        rc = dispatch_k<false>(g, qn, smem_cta, smem_knn, s);
        if (rc) return rc;
        rc = dispatch_knn_list(g, qn, smem_knn, s);
        if (rc) return rc;
      } else {
        // the 27 cells around each central's cell, within the cell edge
        const double rk = (double)g->r_cut * (double)g->cell_scale;
        double e = bins.r0 + (double)bins.n_bins * bins.dr;
        const float Emax = (float)(e * e), Ek = (float)(rk * rk);
        qn.emax_near = Ek < Emax ? Ek : Emax;
        qn.stencil = 1;
        row_widths(1, 1.0, qn.row_w);
        rc = dispatch_k<false>(g, qn, smem_cta, smem_layout(bins.n_bins, n_k, false, 0, true).total, s);
        if (rc) return rc;
        // the full radius for the centrals it marked
        QueryArgs qf = qa;
        qf.fallback = 1;
        qf.need = g->sel;
        qf.next_front = &g->ctr.geo->work_next2b;
        qf.next_light = &g->ctr.geo->work_next3b;
        rc = dispatch_k<false>(g, qf, smem_cta, smem_layout(bins.n_bins, n_k, false, 0, true).total, s);
        if (rc) return rc;
      }
    }
    QueryArgs qs = qa;
    qs.n_k = 0;
    qs.pfx = reinterpret_cast<const uint32_t*>(g->cr);  // written by the central-list compaction
    const uint32_t smem_sym = smem_layout(bins.n_bins, 0, true, 0, true, qa.lut_n).total;
    PS_CUDA(cudaFuncSetAttribute(k_rdf_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sym));
    int per_sm = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rdf_sym, 256, smem_sym));
    if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "symmetric RDF kernel does not fit on an SM");
    PS_LAUNCH(PS_KID_RDF_SYM, s, PS_CUDA(launch_pdl(k_rdf_sym, g->num_sms * per_sm, 256, smem_sym, s, qs)));
  } else if (n_k > 0 || rdf) {
    rc = rdf ? dispatch_k<true>(g, qa, smem_cta, smem_warp, s) : dispatch_k<false>(g, qa, smem_cta, smem_warp, s);
    if (rc) return rc;
  }
  PS_LAUNCH(PS_KID_EPILOGUE, s, PS_CUDA(launch_pdl(k_query_epilogue, 1, 32, 0, s, g->nbr.geo, g->ctr.geo, d_meta)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
