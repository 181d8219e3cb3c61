// Cell-grid binner: counting sort of the ion records into a uniform cell grid.
//
// The paper indexes ions with per-region, per-type KD-trees whose leaves are
// repacked so that the ions of a leaf are contiguous (Suppl. "Details on
// efficient spatial indices"), and uses regular spatial binning for constant
// time queries (Suppl. Fig. QueryingStructures c).  Here the index is the
// regular binning: cells of edge >= r_cut, one set of cells per neighbour
// type set (the paper keeps one tree per ion type, Suppl. "Effectiveness of
// spatial splitting"), records sorted by cell as float4 (x, y, z, index).
//
// Pipeline (all on the device, no host synchronisation):
//   reset -> select + bounding box -> geometry + zero counts -> count ranks
//   -> single-pass exclusive scan (decoupled look-back) -> scatter
// The selection kernels read 16 type labels per thread (one 16-byte load).
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;
constexpr int kGroup = 16;  // ions per thread in the selection kernels

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// warp-aggregated append: returns this lane's slot for lanes with pred set
__device__ __forceinline__ uint32_t warp_append(bool pred, uint32_t* counter) {
  const uint32_t active = __activemask();
  const uint32_t bal = __ballot_sync(active, pred);
  uint32_t base = 0;
  const int leader = __ffs(bal) - 1;
  if (bal != 0 && (int)lane_id() == leader) base = atomicAdd(counter, __popc(bal));
  base = __shfl_sync(active, base, leader < 0 ? 0 : leader);
  return base + __popc(bal & ((1u << lane_id()) - 1u));
}

// warp-aggregated append of `cnt` items per lane (full warp): returns this lane's first slot
__device__ __forceinline__ uint32_t warp_append_n(uint32_t cnt, uint32_t* counter) {
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane_id() >= (uint32_t)o) x += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
  uint32_t base = 0;
  if (lane_id() == 31 && total) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + x - cnt;
}

// block-aggregated append of `cnt` items per thread (every thread of the block
// calls it): one atomic per block instead of one per warp, since appends from
// all warps of the grid to one counter serialise at its L2 slice.  Returns this
// thread's first slot.  s_w and s_x are per-block scratch of blockDim/32 words.
__device__ __forceinline__ uint32_t block_append_n(uint32_t cnt, uint32_t* counter, uint32_t* s_w, uint32_t* s_x,
                                                   uint32_t* s_base) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = lane < nw ? s_w[lane] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    if (lane < nw) s_x[lane] = inc - v;
    if (lane == 31) *s_base = inc ? atomicAdd(counter, inc) : 0u;
  }
  __syncthreads();
  return *s_base + s_x[warp] + x - cnt;
}

// the 16 type labels of group g (ions 16g .. 16g+15); `valid` masks the labels past n
__device__ __forceinline__ void load_types16(const uint8_t* __restrict__ type, int64_t n, int64_t g, bool vec,
                                             uint8_t (&t)[kGroup], uint32_t& valid) {
  const int64_t i0 = g * kGroup;
  const int64_t left = n - i0;
  valid = left >= kGroup ? 0xFFFFu : ((1u << (uint32_t)left) - 1u);
  if (vec && left >= kGroup) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(type + i0));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < kGroup; ++k) t[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
  } else {
#pragma unroll
    for (int k = 0; k < kGroup; ++k) t[k] = (k < left) ? type[i0 + k] : 0;
  }
}

__global__ void k_reset(Geo* geo) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      geo->bbox_key[a] = f2key(INFINITY);
      geo->bbox_key[3 + a] = f2key(-INFINITY);
    }
    geo->n_sel = 0;
    geo->status = 0;
    geo->work_n = geo->work_n2 = geo->work_n3 = geo->work_n4 = 0;
    geo->work_next = geo->work_next2 = geo->work_next3 = 0;
    geo->work_next2b = geo->work_next3b = geo->sym_next = geo->list_n = 0;
  }
}

__device__ __forceinline__ void box_add(float (&lo)[3], float (&hi)[3], bool& bad, float x, float y, float z) {
  if (finite3(x, y, z)) {
    lo[0] = fminf(lo[0], x), hi[0] = fmaxf(hi[0], x);
    lo[1] = fminf(lo[1], y), hi[1] = fmaxf(hi[1], y);
    lo[2] = fminf(lo[2], z), hi[2] = fmaxf(hi[2], z);
  } else {
    bad = true;
  }
}

// Select the ions of the neighbour set, append their indices, reduce the bounding box.
__global__ void __launch_bounds__(kThreads) k_select_bbox(const float* __restrict__ xyz, const uint8_t* __restrict__ type,
                                                          int64_t n, Mask mask, bool vec, uint32_t* __restrict__ sel,
                                                          Geo* geo) {
  griddep_wait();
  griddep_launch();
  __shared__ uint32_t s_aw[kThreads / 32], s_ax[kThreads / 32], s_abase;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  const int64_t groups = (n + kGroup - 1) / kGroup;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < groups; base += stride) {
    const int64_t g = base + threadIdx.x;
    uint32_t m = 0;
    if (g < groups) {
      uint8_t t[kGroup];
      uint32_t valid;
      load_types16(type, n, g, vec, t, valid);
#pragma unroll
      for (int k = 0; k < kGroup; ++k) m |= (in_mask(mask, t[k]) ? 1u : 0u) << k;
      m &= valid;
    }
    const uint32_t cnt = __popc(m);
    uint32_t slot = block_append_n(cnt, &geo->n_sel, s_aw, s_ax, &s_abase);
    const int64_t i0 = g * kGroup;
    if (cnt >= 4 && vec && m == 0xFFFFu) {
      // a full group: read its 192 bytes of coordinates as 12 float4
      const float4* p = reinterpret_cast<const float4*>(xyz + 3 * i0);
      float c[3 * kGroup];
#pragma unroll
      for (int q = 0; q < 3 * kGroup / 4; ++q) {
        const float4 v = __ldg(p + q);
        c[4 * q] = v.x, c[4 * q + 1] = v.y, c[4 * q + 2] = v.z, c[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        box_add(lo, hi, bad, c[3 * k], c[3 * k + 1], c[3 * k + 2]);
        sel[slot + k] = (uint32_t)(i0 + k);
      }
    } else {
      while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        const int64_t i = i0 + k;
        box_add(lo, hi, bad, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
        sel[slot++] = (uint32_t)i;
      }
    }
  }
  // block reduction of the box
  __shared__ float s_lo[3][kThreads / 32], s_hi[3][kThreads / 32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  __syncthreads();
  if (bad) s_bad = 1;
  if (lane_id() == 0)
    for (int a = 0; a < 3; ++a) s_lo[a][threadIdx.x >> 5] = lo[a], s_hi[a][threadIdx.x >> 5] = hi[a];
  __syncthreads();
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    float l = INFINITY, h = -INFINITY;
    for (int w = 0; w < kThreads / 32; ++w) l = fminf(l, s_lo[a][w]), h = fmaxf(h, s_hi[a][w]);
    if (l <= h) {
      atomicMin(&geo->bbox_key[a], f2key(l));
      atomicMax(&geo->bbox_key[3 + a], f2key(h));
    }
  }
  if (threadIdx.x == 0 && s_bad) atomicCAS(&geo->status, 0, (int)PS_ERR_INVALID_INPUT);
}

// Cell geometry from the bounding box.  The cell edge carries a margin so that
// every pair within r_cut lies within `stencil` cells of each other despite
// float32 rounding of the cell index: stencil * h >= r_cut * (1 + 2^-10) +
// extent * 2^-20 (cell_scale >= 1/stencil).
__device__ void compute_geometry(const Geo& in, float r_cut, float cell_scale, uint32_t cell_cap, Geo& out) {
  double lo[3], hi[3];
  const bool empty = in.n_sel == 0 || in.bbox_key[0] > in.bbox_key[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = empty ? 0.0 : (double)key2f(in.bbox_key[a]);
    hi[a] = empty ? 0.0 : (double)key2f(in.bbox_key[3 + a]);
  }
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = fmax(ext, hi[a] - lo[a]);
  double h = (double)r_cut * (double)cell_scale * (1.0 + 1.0 / 1024.0) + ext * (1.0 / 1048576.0);
  uint32_t dims[3] = {1, 1, 1};
  // cells smaller than r_cut: room in the cell arrays for the grid of cells centred on the
  // vertices (one more cell per axis) that the query in passes sorts its centrals by
  const double extra = cell_scale < 1.0f ? 1.0 : 0.0;
  for (int it = 0; it < 256; ++it) {
    double tot = 1.0;
    for (int a = 0; a < 3; ++a) {
      double d = floor((hi[a] - lo[a]) / h) + 1.0;
      d = fmin(d, 2147483648.0);
      dims[a] = (uint32_t)d;
      tot *= d + extra;
    }
    if (tot <= (double)cell_cap) break;
    h *= 1.2599210498948732;  // 2^(1/3): halve the cell count
  }
  for (int a = 0; a < 3; ++a) {
    out.origin[a] = (float)lo[a];
    out.dims[a] = dims[a];
  }
  out.h = (float)h;
  out.inv_h = (float)(1.0 / h);
  out.n_cells = dims[0] * dims[1] * dims[2];
}

// One thread per block computes the geometry; block 0 publishes it; all zero the counts.
__global__ void __launch_bounds__(kThreads) k_geometry_zero(Geo* geo, float r_cut, float cell_scale, uint32_t cell_cap,
                                                            uint32_t* __restrict__ count) {
  griddep_wait();
  griddep_launch();
  __shared__ uint32_t s_nc;
  if (threadIdx.x == 0) {
    Geo g = *geo;
    compute_geometry(g, r_cut, cell_scale, cell_cap, g);
    s_nc = g.n_cells;
    if (blockIdx.x == 0) {
      for (int a = 0; a < 3; ++a) geo->origin[a] = g.origin[a], geo->dims[a] = g.dims[a];
      geo->h = g.h;
      geo->inv_h = g.inv_h;
      geo->n_cells = g.n_cells;
    }
  }
  __syncthreads();
  const uint32_t nc = s_nc;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) count[c] = 0;
}

// Cell index and rank (arrival order within the cell) of every selected ion.
__global__ void __launch_bounds__(kThreads) k_count(const float* __restrict__ xyz, const uint32_t* __restrict__ sel,
                                                    const Geo* __restrict__ geo, uint32_t* __restrict__ count,
                                                    uint2* __restrict__ cr) {
  griddep_wait();
  griddep_launch();
  const Geo g = *geo;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < g.n_sel; s += gridDim.x * blockDim.x) {
    const uint32_t i = sel[s];
    const uint32_t c = cell_of(g, xyz[3 * (int64_t)i], xyz[3 * (int64_t)i + 1], xyz[3 * (int64_t)i + 2]);
    cr[s] = make_uint2(c, atomicAdd(&count[c], 1u));
  }
}

// Central ions: type in mask and d_srf >= dsrf_min, binned into the neighbour geometry.
__global__ void __launch_bounds__(kThreads) k_central_select_count(const float* __restrict__ xyz,
                                                                   const uint8_t* __restrict__ type,
                                                                   const float* __restrict__ dsrf, int64_t n, Mask mask,
                                                                   float dsrf_min, bool vec, const Geo* __restrict__ ngeo,
                                                                   Geo* cgeo, uint32_t* __restrict__ count,
                                                                   uint32_t* __restrict__ sel, uint2* __restrict__ cr) {
  griddep_wait();
  griddep_launch();
  __shared__ uint32_t s_aw[kThreads / 32], s_ax[kThreads / 32], s_abase;
  const Geo g = *ngeo;
  bool bad = false;
  const int64_t groups = (n + kGroup - 1) / kGroup;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < groups; base += stride) {
    const int64_t gi = base + threadIdx.x;
    uint32_t m = 0;
    const int64_t i0 = gi * kGroup;
    if (gi < groups) {
      uint8_t t[kGroup];
      uint32_t valid;
      load_types16(type, n, gi, vec, t, valid);
#pragma unroll
      for (int k = 0; k < kGroup; ++k) m |= (in_mask(mask, t[k]) ? 1u : 0u) << k;
      m &= valid;
      if (dsrf != nullptr && m) {
        uint32_t keep = 0;
        if (m == 0xFFFFu && vec) {
          const float4* p = reinterpret_cast<const float4*>(dsrf + i0);
#pragma unroll
          for (int q = 0; q < kGroup / 4; ++q) {
            const float4 v = __ldg(p + q);
            keep |= ((v.x >= dsrf_min) ? 1u : 0u) << (4 * q);
            keep |= ((v.y >= dsrf_min) ? 1u : 0u) << (4 * q + 1);
            keep |= ((v.z >= dsrf_min) ? 1u : 0u) << (4 * q + 2);
            keep |= ((v.w >= dsrf_min) ? 1u : 0u) << (4 * q + 3);
          }
        } else {
          uint32_t mm = m;
          while (mm) {
            const int k = __ffs(mm) - 1;
            mm &= mm - 1;
            keep |= ((dsrf[i0 + k] >= dsrf_min) ? 1u : 0u) << k;
          }
        }
        m &= keep;
      }
    }
    uint32_t slot = block_append_n(__popc(m), &cgeo->n_sel, s_aw, s_ax, &s_abase);
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1;
      const int64_t i = i0 + k;
      const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
      bad |= !finite3(x, y, z);
      const uint32_t c = cell_of(g, x, y, z);
      sel[slot] = (uint32_t)i;
      cr[slot] = make_uint2(c, atomicAdd(&count[c], 1u));
      ++slot;
    }
  }
  if (bad) atomicCAS(&cgeo->status, 0, (int)PS_ERR_INVALID_INPUT);
}

// Resets the central list (copies the neighbour geometry, zeroes the counters
// and cell counts) and zeroes the query's output arrays.
__global__ void k_central_reset(const Geo* __restrict__ ngeo, Geo* cgeo, uint32_t* __restrict__ count, ZeroOut z) {
  griddep_wait();
  griddep_launch();
  const uint32_t nc = ngeo->n_cells;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cgeo = *ngeo;
    cgeo->n_sel = 0;
    cgeo->status = 0;
    cgeo->work_n = cgeo->work_n2 = cgeo->work_n3 = cgeo->work_n4 = 0;
    cgeo->work_next = cgeo->work_next2 = cgeo->work_next3 = 0;
    cgeo->work_next2b = cgeo->work_next3b = cgeo->sym_next = cgeo->list_n = 0;
  }
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (uint32_t c = tid; c < nc; c += stride) count[c] = 0;
  for (int k = 0; k < 3; ++k)
    if (z.p[k])
      for (uint32_t i = tid; i < z.n[k]; i += stride) z.p[k][i] = 0ull;
}

// ---- exclusive scan of the cell counts ------------------------------------

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t prefix = warp ? s_warp[warp - 1] : 0u;
  total = s_warp[nw - 1];
  __syncthreads();
  return prefix + x - v;
}

// Candidates of cell c: the neighbour records in the cells within `st` (1 or 2) cells of it.
// The row loops are unrolled over the largest stencil so that the loads issue together.
__device__ __forceinline__ uint32_t stencil_count(const uint32_t* __restrict__ nstart, const Geo* g, uint32_t c, int st) {
  const uint32_t d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const uint32_t cx = c % d0, cy = (c / d0) % d1, cz = c / (d0 * d1);
  const uint32_t xlo = cx >= (uint32_t)st ? cx - st : 0, xhi = cx + st < d0 ? cx + st : d0 - 1;
  uint32_t n = 0;
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy) {
      const int z = (int)cz + dz, y = (int)cy + dy;
      if (dz >= -st && dz <= st && dy >= -st && dy <= st && z >= 0 && y >= 0 && z < (int)d2 && y < (int)d1) {
        const uint32_t row = ((uint32_t)z * d1 + (uint32_t)y) * d0;
        n += __ldg(nstart + row + xhi + 1) - __ldg(nstart + row + xlo);
      }
    }
  return n;
}

// Warp items of a cell with n centrals: n <= 3 gives one item (the lanes of
// the warp split the candidates of each central); otherwise ceil(n/32)
// batches of at most 32 centrals (one lane per central).  With L lanes per
// central an item holds at most 32 / L centrals.  Balanced batches for the
// kernels that give every central one lane; for the exact query (`split`)
// full batches of 32 / L and one remainder, whose centrals then get
// item_lanes(remainder) lanes each.
__device__ __forceinline__ uint32_t items_of(uint32_t n, uint32_t L = 1) {
  const uint32_t per = 32u / L;
  return n == 0 ? 0u : (n <= 3 ? 1u : (n + per - 1u) / per);
}

// look-back words: flag in bits 62-63 (1: tile aggregate, 2: inclusive prefix), value in bits 0-31
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62;

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Warp 0 of the CTA that owns scan tile t (tiles are numbered in the order CTAs
// claim them, so every tile it looks back at belongs to a CTA that is already
// running or done): publishes the tile's aggregate, looks back 32 predecessors
// at a time (lane l reads tile j - l; the window is summed up to the nearest tile
// that holds an inclusive prefix; the virtual tile -1 holds prefix 0), publishes
// the inclusive prefix and returns the exclusive one in every lane.  A wait on a
// predecessor gives up after limit_ns and records PS_ERR_TIMEOUT in *status.
__device__ uint32_t tile_lookback(uint32_t t, uint32_t total, unsigned long long* state, int* status,
                                  uint64_t limit_ns = kWaitLimitNs) {
  const uint32_t lane = lane_id();
  uint32_t prefix = 0;
  if (t > 0) {
    if (lane == 0) st_release(&state[t], kFlagA | total);
    int j = (int)t - 1;
    uint64_t t0 = 0;
    while (j >= 0) {
      const int idx = j - (int)lane;
      const unsigned long long w = idx >= 0 ? ld_acquire(&state[idx]) : kFlagP;
      const uint32_t isP = __ballot_sync(0xffffffffu, (w >> 62) == 2);
      const uint32_t notready = __ballot_sync(0xffffffffu, (w >> 62) == 0);
      const uint32_t lim = isP ? (uint32_t)(__ffs(isP) - 1) : 31u;
      const uint32_t need = lim == 31u ? 0xffffffffu : ((2u << lim) - 1u);
      if (notready & need) {
        int give_up = 0;
        if (lane == 0) {
          if (t0 == 0) t0 = global_ns();
          give_up = global_ns() - t0 > limit_ns;
        }
        if (__shfl_sync(0xffffffffu, give_up, 0)) {
          if (lane == 0) atomicCAS(status, 0, (int)PS_ERR_TIMEOUT);
          break;
        }
        continue;
      }
      uint32_t v = lane <= lim ? (uint32_t)w : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      prefix += v;
      if (isP) break;
      j -= 32;
      t0 = 0;
    }
  }
  if (lane == 0) st_release(&state[t], kFlagP | (uint32_t)(prefix + total));
  return prefix;
}

// End of a single-pass scan (thread 0 of every CTA): the last CTA to finish clears
// the look-back words and the tile counter for the next scan.
__device__ void scan_finish(unsigned long long* state, uint32_t* ctr, uint32_t tiles) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctr[1], 1u) == gridDim.x - 1) {
      for (uint32_t i = 0; i < tiles; ++i) state[i] = 0ull;
      ctr[0] = 0;
      __threadfence();
      ctr[1] = 0;
    }
  }
}

// Work lists of the central list for the kScanItems cells c0.. with v[k] centrals
// (every lane of the warp calls it): cells with at least dense_min centrals go to
// `work` (CTA kernel), the others are split into warp items (cell,
// first << 6 | count): sparse cells (fewer than kHeavy centrals and at most
// kSparseCand candidates in the stencil of the neighbour grid `nstart`) from the
// back of `witem`, the rest from the front.  With `split` (the exact query),
// batches of 32 / lanes_per_central centrals and one remainder, and the very heavy
// items (very_heavy) in `whi` instead of the front of `witem`; otherwise balanced
// batches of at most 32.
__device__ __forceinline__ void emit_items(const uint32_t (&v)[kScanItems], uint32_t c0, uint32_t nc, Geo* geo,
                                           uint32_t* __restrict__ work, uint2* __restrict__ witem, uint32_t dense_min,
                                           uint32_t cap, const uint32_t* __restrict__ nstart, int stencil, bool split,
                                           uint2* __restrict__ whi) {
  uint32_t n_front = 0, n_back = 0, n_hi = 0;
  // the work-shape estimates count the candidates of at most 5 x 5 rows (the 7 x 7 rows of a
  // three-cell stencil would double the loads of this scan for a heuristic)
  stencil = stencil > 2 ? 2 : stencil;
  bool sparse[kScanItems];
  uint32_t lanes[kScanItems], cands[kScanItems];
  const uint32_t n_nbr = nstart != nullptr ? nstart[nc] : 0u;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const bool dense = (c0 + k < nc) && v[k] >= dense_min;
    const uint32_t s1 = warp_append(dense, &geo->work_n);
    if (dense) work[s1] = c0 + k;
    const uint32_t cand = (!dense && v[k] > 0 && nstart != nullptr) ? stencil_count(nstart, geo, c0 + k, stencil) : 0u;
    sparse[k] = !dense && v[k] > 0 && v[k] < kHeavy && nstart != nullptr && cand <= kSparseCand;
    lanes[k] = (split && nstart != nullptr && !sparse[k] && v[k] > 3) ? lanes_per_central(cand, n_nbr, nc, stencil)
                                                                        : 1u;
    cands[k] = cand;
    if (!dense && sparse[k]) n_back += items_of(v[k], lanes[k]);
    if (!dense && !sparse[k]) {
      const uint32_t m = items_of(v[k], lanes[k]), per = 32u / lanes[k];
      for (uint32_t q = 0, first = 0; q < m; ++q) {
        const uint32_t cnt = split ? min(per, v[k] - first) : 0u;
        const bool hi = whi != nullptr && cnt > 3 && very_heavy(cand, item_lanes(cnt), n_nbr, nc, stencil);
        (hi ? n_hi : n_front) += 1;
        first += cnt;
      }
    }
  }
  uint32_t hs = warp_append_n(n_front, &geo->work_n2);
  uint32_t ls = warp_append_n(n_back, &geo->work_n3);
  uint32_t xs = warp_append_n(n_hi, &geo->work_n4);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (v[k] >= dense_min) continue;
    const uint32_t m = items_of(v[k], lanes[k]);
    if (m == 0) continue;
    const uint32_t base = v[k] / m, rem = v[k] % m, per = 32u / lanes[k];
    uint32_t first = 0;
    for (uint32_t q = 0; q < m; ++q) {
      const uint32_t cnt = split ? min(per, v[k] - first) : base + (q < rem ? 1u : 0u);
      const uint2 it = make_uint2(c0 + k, (first << 6) | cnt);
      if (sparse[k])
        witem[cap - 1 - ls++] = it;
      else if (whi != nullptr && split && cnt > 3 && very_heavy(cands[k], item_lanes(cnt), n_nbr, nc, stencil))
        whi[xs++] = it;
      else
        witem[hs++] = it;
      first += cnt;
    }
  }
}

// Single-pass exclusive scan of the cell counts (decoupled look-back).  Also
// writes the end sentinel and, for the central list (`work` given), the work
// lists (emit_items).
__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t* __restrict__ count, Geo* geo,
                                                       uint32_t* __restrict__ start, uint32_t* __restrict__ work,
                                                       uint2* __restrict__ witem, uint32_t dense_min, uint32_t cap,
                                                       unsigned long long* state, uint32_t* ctr,
                                                       const uint32_t* __restrict__ nstart, int stencil, bool split,
                                                       uint2* __restrict__ whi) {
  griddep_wait();
  griddep_launch();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_tile, s_prefix;
  const uint32_t nc = geo->n_cells;
  const uint32_t tiles = (nc + kScanTile - 1) / kScanTile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= tiles) break;
    const uint32_t c0 = t * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (c0 + k < nc) ? count[c0 + k] : 0u;
      sum += v[k];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x < 32) {
      const uint32_t prefix = tile_lookback(t, total, state, &geo->status);
      if (lane_id() == 0) {
        s_prefix = prefix;
        if (t == tiles - 1) start[nc] = prefix + total;  // end sentinel: number of records
      }
    }
    __syncthreads();
    uint32_t run = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (c0 + k < nc) start[c0 + k] = run;
      run += v[k];
    }
    if (work != nullptr) emit_items(v, c0, nc, geo, work, witem, dense_min, cap, nstart, stencil, split, whi);
    __syncthreads();  // s_tile and s_prefix are rewritten next
  }
  scan_finish(state, ctr, tiles);
}

// Central list of a central type set contained in the neighbour set, step 1 of 2.
// The centrals are then a subset of the neighbour records, which are already
// sorted by cell: an order-preserving compaction of those records (single-pass
// scan of the central flags over the records) gives the sorted central records
// directly, with no second pass over the whole cloud and no counting sort.  pfx[j]
// = number of centrals among records 0..j-1 (pfx[n_records] = all), from which
// k_central_items reads the cell starts.  Also resets the central list's geometry
// and counters and zeroes the query's outputs.
__global__ void __launch_bounds__(kScanThreads) k_central_subset(const float4* __restrict__ nrec,
                                                                 const Geo* __restrict__ ngeo, Geo* cgeo,
                                                                 const uint8_t* __restrict__ type,
                                                                 const float* __restrict__ dsrf, Mask mask,
                                                                 float dsrf_min, float4* __restrict__ crec,
                                                                 uint32_t* __restrict__ pfx, unsigned long long* state,
                                                                 uint32_t* ctr, ZeroOut z, uint32_t* __restrict__ vcount) {
  griddep_wait();
  griddep_launch();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_tile, s_prefix;
  const uint32_t nr = ngeo->n_sel;
  // vcount given: the central list is the grid of cells centred on the vertices (origin half a
  // cell lower, one more cell per axis), filled by k_vertex_count / k_vertex_scatter; its counts
  // are zeroed here and no records are written
  const uint32_t nvc = (ngeo->dims[0] + 1) * (ngeo->dims[1] + 1) * (ngeo->dims[2] + 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // every field but n_sel, which the thread that scans the last tile writes
    const float half = vcount ? __fmul_rn(0.5f, ngeo->h) : 0.0f;
    for (int a = 0; a < 3; ++a)
      cgeo->origin[a] = __fsub_rn(ngeo->origin[a], half), cgeo->dims[a] = ngeo->dims[a] + (vcount ? 1u : 0u);
    for (int a = 0; a < 6; ++a) cgeo->bbox_key[a] = ngeo->bbox_key[a];
    cgeo->inv_h = ngeo->inv_h;
    cgeo->h = ngeo->h;
    cgeo->n_cells = vcount ? nvc : ngeo->n_cells;
    cgeo->status = 0;
    cgeo->work_n = cgeo->work_n2 = cgeo->work_n3 = cgeo->work_n4 = 0;
    cgeo->work_next = cgeo->work_next2 = cgeo->work_next3 = 0;
    cgeo->work_next2b = cgeo->work_next3b = cgeo->sym_next = cgeo->list_n = 0;
    if (nr == 0) pfx[0] = 0, cgeo->n_sel = 0;
  }
  {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int k = 0; k < 3; ++k)
      if (z.p[k])
        for (uint32_t i = tid; i < z.n[k]; i += stride) z.p[k][i] = 0ull;
    if (vcount)
      for (uint32_t i = tid; i < nvc; i += stride) vcount[i] = 0u;
  }
  const uint32_t tiles = (nr + kScanTile - 1) / kScanTile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= tiles) break;
    const uint32_t j0 = t * kScanTile + threadIdx.x * kScanItems;
    float4 r[kScanItems];
    uint32_t f[kScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      f[k] = 0;
      if (j0 + k < nr) {
        r[k] = nrec[j0 + k];
        const uint32_t idx = __float_as_uint(r[k].w);
        f[k] = (in_mask(mask, type[idx]) && (dsrf == nullptr || dsrf[idx] >= dsrf_min)) ? 1u : 0u;
      }
      sum += f[k];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x < 32) {
      const uint32_t prefix = tile_lookback(t, total, state, &cgeo->status);
      if (lane_id() == 0) {
        s_prefix = prefix;
        if (t == tiles - 1) pfx[nr] = prefix + total, cgeo->n_sel = prefix + total;
      }
    }
    __syncthreads();
    uint32_t run = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (j0 + k < nr) {
        pfx[j0 + k] = run;
        if (f[k] && crec) crec[run] = r[k];
      }
      run += f[k];
    }
    __syncthreads();  // s_tile and s_prefix are rewritten next
  }
  scan_finish(state, ctr, tiles);
}

// Central list of a central type set contained in the neighbour set, step 2 of 2:
// cell starts from the record prefix (a cell's centrals are the flagged records
// among its neighbour records), the end sentinel and the work lists.
__global__ void __launch_bounds__(kThreads) k_central_items(const uint32_t* __restrict__ nstart,
                                                            const uint32_t* __restrict__ pfx, Geo* cgeo,
                                                            uint32_t* __restrict__ start, uint32_t* __restrict__ work,
                                                            uint2* __restrict__ witem, uint32_t dense_min, uint32_t cap,
                                                            int stencil, bool split, uint2* __restrict__ whi) {
  griddep_wait();
  griddep_launch();
  const uint32_t nc = cgeo->n_cells;
  // after a look-back that gave up (status set) the prefixes may be inconsistent: no work items
  const bool ok = cgeo->status == 0;
  const uint32_t step = gridDim.x * blockDim.x * kScanItems;
  // the loop bound is uniform per block: every lane reaches the warp-wide appends
  for (uint32_t base = blockIdx.x * blockDim.x * kScanItems; base < nc; base += step) {
    const uint32_t c0 = base + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = 0;
      const uint32_t c = c0 + k;
      if (c < nc) {
        const uint32_t b = pfx[nstart[c]], e = pfx[nstart[c + 1]];
        start[c] = b;
        v[k] = (ok && e >= b) ? e - b : 0u;
        if (c == nc - 1) start[nc] = e;
      }
    }
    emit_items(v, c0, nc, cgeo, work, witem, dense_min, cap, nstart, stencil, split, whi);
  }
}

// Central list on the vertex-centred grid (cgeo: origin half a cell below the neighbour grid's,
// one more cell per axis), for the query in passes: the centrals of the cell around vertex V are
// those nearest to V, and the 2 x 2 x 2 neighbour cells around V hold every record within half a
// cell of each of them.  Counting sort of the flagged neighbour records (pfx), in the record
// order: count + rank here, starts by k_scan, records by k_vertex_scatter.
__global__ void __launch_bounds__(kThreads) k_vertex_count(const float4* __restrict__ nrec,
                                                           const Geo* __restrict__ ngeo, const Geo* __restrict__ cgeo,
                                                           const uint32_t* __restrict__ pfx,
                                                           uint32_t* __restrict__ count, uint32_t* __restrict__ rank) {
  griddep_wait();
  griddep_launch();
  const uint32_t nr = ngeo->n_sel;
  const Geo g = *cgeo;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
    const uint32_t c0 = pfx[j];
    if (pfx[j + 1] == c0) continue;
    const float4 p = nrec[j];
    rank[c0] = atomicAdd(&count[cell_of(g, p.x, p.y, p.z)], 1u);
  }
}

__global__ void __launch_bounds__(kThreads) k_vertex_scatter(const float4* __restrict__ nrec,
                                                             const Geo* __restrict__ ngeo,
                                                             const Geo* __restrict__ cgeo,
                                                             const uint32_t* __restrict__ pfx,
                                                             const uint32_t* __restrict__ start,
                                                             const uint32_t* __restrict__ rank,
                                                             float4* __restrict__ crec) {
  griddep_wait();
  griddep_launch();
  const uint32_t nr = ngeo->n_sel;
  const Geo g = *cgeo;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
    const uint32_t c0 = pfx[j];
    if (pfx[j + 1] == c0) continue;
    const float4 p = nrec[j];
    crec[start[cell_of(g, p.x, p.y, p.z)] + rank[c0]] = p;
  }
}

// Scatter the selected ions to their sorted slot.  The record's 4th word is the
// ion index, or (index << 8 | type) when `type` is given (clouds of < 2^24 ions).
__global__ void __launch_bounds__(kThreads) k_scatter(const float* __restrict__ xyz, const uint32_t* __restrict__ sel,
                                                      const uint2* __restrict__ cr, const uint32_t* __restrict__ start,
                                                      const Geo* __restrict__ cnt, float4* __restrict__ rec,
                                                      const uint8_t* __restrict__ type) {
  griddep_wait();
  griddep_launch();
  const uint32_t ns = cnt->n_sel;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const uint32_t i = sel[s];
    const uint2 c = cr[s];
    const int64_t b = 3 * (int64_t)i;
    const uint32_t w = type ? ((i << 8) | type[i]) : i;
    rec[start[c.x] + c.y] = make_float4(xyz[b], xyz[b + 1], xyz[b + 2], __uint_as_float(w));
  }
}

// Self-test of the two bounded waits of the library on events that never happen
// (one warp): the look-back of a scan tile whose predecessor never publishes, and
// an mbarrier phase that nothing completes.  Each must give up after limit_ns and
// report PS_ERR_TIMEOUT; nothing is in flight when the kernel returns.
//   work[0], work[1]  look-back words of tiles 0 and 1 (tile 0 stays unpublished)
//   work[2]           status of the look-back wait (low 32 bits)
//   work[3]           status of the mbarrier wait
__global__ void k_wait_selftest(unsigned long long* work, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    work[0] = 0ull;
    work[1] = 0ull;
    work[2] = 0ull;
    work[3] = 0ull;
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __threadfence();
  __syncwarp();
  tile_lookback(1, 0, work, reinterpret_cast<int*>(work + 2), limit_ns);
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) work[3] = (unsigned long long)PS_ERR_TIMEOUT;
}

int wait_selftest(uint64_t limit_ns, unsigned long long* d_work, cudaStream_t s) {
  PS_LAUNCH(PS_KID_SCAN, s, k_wait_selftest<<<1, 32, 0, s>>>(d_work, limit_ns));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

static int grid_blocks(const ps_grid* g, int per_sm) { return g->num_sms * per_sm; }

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static int scan_cells(ps_grid* g, CellList& L, Geo* geo, bool with_work, cudaStream_t s, bool split = false) {
  PS_LAUNCH(PS_KID_SCAN, s,
            PS_CUDA(launch_pdl(k_scan, grid_blocks(g, 1), kScanThreads, 0, s, L.count, geo, L.start, with_work ? L.work : nullptr,
                                                               L.witem, g->dense_min, g->item_cap, g->scan_state,
                                                               g->scan_ctr, with_work ? g->nbr.start : nullptr,
                                                               g->stencil, split, split ? g->nbr_witem : nullptr)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int build_neighbour_grid(ps_grid* g, const uint64_t nbr_mask[4], float r_cut, cudaStream_t s) {
  Mask m;
  for (int w = 0; w < 4; ++w) m.w[w] = nbr_mask[w], g->nbr_mask[w] = nbr_mask[w];
  Geo* geo = g->nbr.geo;
  const bool vec = aligned16(g->type) && aligned16(g->xyz);
  PS_LAUNCH(PS_KID_RESET, s, PS_CUDA(launch_pdl(k_reset, 1, 32, 0, s, geo)));
  if (g->n > 0)
    PS_LAUNCH(PS_KID_SELECT, s,
              PS_CUDA(launch_pdl(k_select_bbox, grid_blocks(g, 8), kThreads, 0, s, g->xyz, g->type, g->n, m, vec, g->sel, geo)));
  PS_LAUNCH(PS_KID_GEOMETRY, s,
            PS_CUDA(launch_pdl(k_geometry_zero, grid_blocks(g, 4), kThreads, 0, s, geo, r_cut, g->cell_scale, g->cell_cap, g->nbr.count)));
  PS_LAUNCH(PS_KID_COUNT, s, PS_CUDA(launch_pdl(k_count, grid_blocks(g, 8), kThreads, 0, s, g->xyz, g->sel, geo, g->nbr.count, g->cr)));
  int rc = scan_cells(g, g->nbr, geo, false, s);
  if (rc) return rc;
  PS_LAUNCH(PS_KID_SCATTER, s,
            PS_CUDA(launch_pdl(k_scatter, grid_blocks(g, 8), kThreads, 0, s, g->xyz, g->sel, g->cr, g->nbr.start, geo, g->nbr.rec,
                                                             g->pack_type ? g->type : nullptr)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int build_central_list(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, cudaStream_t s,
                       ZeroOut z, bool split, bool vertex) {
  Mask m;
  bool subset = !g->pack_type;
  for (int w = 0; w < 4; ++w) m.w[w] = ctr_mask[w], subset = subset && (ctr_mask[w] & ~g->nbr_mask[w]) == 0;
  if (subset && vertex) {
    // the central prefix over the neighbour records, then the centrals sorted by the
    // vertex-centred grid (ranks in the dense-cell list, unused without dense cells)
    uint32_t* pfx = reinterpret_cast<uint32_t*>(g->cr);
    PS_LAUNCH(PS_KID_CENTRAL, s,
              PS_CUDA(launch_pdl(k_central_subset, grid_blocks(g, 1), kScanThreads, 0, s, g->nbr.rec, g->nbr.geo,
                                 g->ctr.geo, g->type, dsrf, m, dsrf_min, (float4*)nullptr, pfx, g->scan_state,
                                 g->scan_ctr, z, g->ctr.count)));
    PS_LAUNCH(PS_KID_CENTRAL, s,
              PS_CUDA(launch_pdl(k_vertex_count, grid_blocks(g, 8), kThreads, 0, s, g->nbr.rec, g->nbr.geo, g->ctr.geo,
                                 pfx, g->ctr.count, g->ctr.work)));
    PS_LAUNCH(PS_KID_SCAN, s,
              PS_CUDA(launch_pdl(k_scan, grid_blocks(g, 1), kScanThreads, 0, s, g->ctr.count, g->ctr.geo, g->ctr.start,
                                 g->ctr.work, g->ctr.witem, 0xFFFFFFFFu, g->item_cap, g->scan_state, g->scan_ctr,
                                 (const uint32_t*)nullptr, g->stencil, true, (uint2*)nullptr)));
    PS_LAUNCH(PS_KID_SCATTER, s,
              PS_CUDA(launch_pdl(k_vertex_scatter, grid_blocks(g, 8), kThreads, 0, s, g->nbr.rec, g->nbr.geo,
                                 g->ctr.geo, pfx, g->ctr.start, g->ctr.work, g->ctr.rec)));
    PS_CUDA(cudaGetLastError());
    return PS_OK;
  }
  if (subset) {
    // centrals are neighbour records: compact the cell-sorted records (2 kernels)
    uint32_t* pfx = reinterpret_cast<uint32_t*>(g->cr);  // 2 n_max words, n_records + 1 needed
    PS_LAUNCH(PS_KID_CENTRAL, s,
              PS_CUDA(launch_pdl(k_central_subset, grid_blocks(g, 1), kScanThreads, 0, s, g->nbr.rec, g->nbr.geo,
                                 g->ctr.geo, g->type, dsrf, m, dsrf_min, g->ctr.rec, pfx, g->scan_state, g->scan_ctr, z,
                                 (uint32_t*)nullptr)));
    PS_LAUNCH(PS_KID_SCAN, s,
              PS_CUDA(launch_pdl(k_central_items, grid_blocks(g, 4), kThreads, 0, s, g->nbr.start, pfx, g->ctr.geo,
                                 g->ctr.start, g->ctr.work, g->ctr.witem, g->dense_min, g->item_cap, g->stencil, split,
                                 split ? g->nbr_witem : nullptr)));
    PS_CUDA(cudaGetLastError());
    return PS_OK;
  }
  const bool vec = aligned16(g->type) && aligned16(g->xyz) && (dsrf == nullptr || aligned16(dsrf));
  PS_LAUNCH(PS_KID_CENTRAL, s,
            PS_CUDA(launch_pdl(k_central_reset, grid_blocks(g, 4), kThreads, 0, s, g->nbr.geo, g->ctr.geo, g->ctr.count, z)));
  if (g->n > 0)
    PS_LAUNCH(PS_KID_CENTRAL, s,
              PS_CUDA(launch_pdl(k_central_select_count, grid_blocks(g, 8), kThreads, 0, s, g->xyz, g->type, dsrf, g->n, m, dsrf_min,
                                                                              vec, g->nbr.geo, g->ctr.geo, g->ctr.count,
                                                                              g->sel, g->cr)));
  int rc = scan_cells(g, g->ctr, g->ctr.geo, true, s, split);
  if (rc) return rc;
  PS_LAUNCH(PS_KID_SCATTER, s,
            PS_CUDA(launch_pdl(k_scatter, grid_blocks(g, 8), kThreads, 0, s, g->xyz, g->sel, g->cr, g->ctr.start, g->ctr.geo, g->ctr.rec,
                                                             g->pack_type ? g->type : nullptr)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
