// Gaussian-smoothed RDF and its adjoint (the differentiable form).
//
// The paper bins pair distances with rectangular transfer functions (Methods,
// "Descriptive, two-point spatial statistics, and clustering").  Here every
// pair spreads a Gaussian of width sigma that is integrated over each bin:
//   u_ij = s * |x_j - x_i|,  K_b(u) = Phi((e_{b+1} - u)/sigma) - Phi((e_b - u)/sigma)
//   h[b] = sum over central i, neighbour j != i with u_ij < stop + 6 sigma of K_b(u_ij)
// and, for an upstream gradient G[b] = dL/dh[b],
//   W(u) = dL/du = sum_b G[b] K_b'(u),
//   dL/dx_i += W s (x_i - x_j)/d,  dL/dx_j -= W s (x_i - x_j)/d,  dL/ds += W d.
//
// Forward: each pair deposits u on a fine grid of width w (<= sigma/40) as three
// moments about the fine-bin centre c_m (count, sum of delta, sum of delta^2);
// a finalize kernel evaluates h[b] = sum_m M0 K_b(c_m) + M1 K_b'(c_m) + M2/2 K_b''(c_m)
// in FP64 over all bins.  The remainder is third order in delta (|delta| <= w/2)
// and odd about c_m, i.e. a relative error ~1e-7 that averages out.
// Adjoint: W, W', W'' are tabulated on the same fine grid (FP64, stored as
// float) and evaluated per pair by the same second-order expansion.  Pairs are
// recomputed, never stored.  Record k's gradient gathers every pair it is in,
// W s (x_k - x_m)/d, once for each role: as the central (m a neighbour) and as
// the neighbour (m a central).  When the centrals are neighbour records, one
// pass has every neighbour record own its gradient, with the pair weighted by
// the central flags of both ends (0, 1 or 2); otherwise pass A (one lane per
// central) writes and pass B (one lane per neighbour, candidates = centrals)
// adds.  Each gradient has one owner: no atomics on the gradient.  dL/ds sums
// W d over the pairs with a central owner.
// Both kernels test the candidates two at a time with packed float32.  The
// forward over unordered pairs takes the neighbour cells one by one: the half
// stencil's records are the lanes and the cell's records are read from shared
// memory by every lane at once; the in-range pairs are compacted into a warp
// list that all lanes bin.  The adjoint runs the pair code under a branch per
// candidate (its per-pair work needs the owner's accumulators).
#include <cmath>
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

constexpr int kSoftRuns = 49;  // (2 * stencil + 1)^2 for stencil <= 3

struct SoftArgs {
  // owners (one lane per record) and their work items
  const float4* orec;
  const uint32_t* ostart;
  const uint2* oitem;
  uint32_t ocap;    // capacity of oitem
  Geo* ogeo;        // owner list counters (work_n2 + work_n3 items, work_next2)
  // candidates and their cell starts (same geometry as the owners)
  const float4* nrec;
  const uint32_t* nstart;
  const Geo* ngeo;  // geometry
  int stencil;
  float scale, sigma, rc;  // rc = stop + 6 sigma (scaled units)
  float rc2u;              // (rc / scale)^2 * (1 + 1e-6): cheap prefilter on d2
  float w, inv_w;          // fine grid
  uint32_t n_fine;
  // forward outputs
  unsigned long long* M0;
  double* M1;
  double* M2;
  // adjoint
  const float* T;          // [3][n_fine]: W, W', W'' at the fine-bin centres
  const uint32_t* pfx;     // one-pass adjoint: central prefix over the neighbour records
  float* grad;             // [n][3]
  double* grad_s;
  int pass_b;              // 0: owners are centrals (write), 1: owners are neighbours (add, sign flipped)
};

__device__ __forceinline__ void soft_run(const SoftArgs& a, const Geo& ng, uint32_t c, uint32_t r, uint32_t& src,
                                         uint32_t& len) {
  const int s = a.stencil, wd = 2 * s + 1;
  const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
  const int y = (int)cy + (int)(r % wd) - s, z = (int)cz + (int)(r / wd) - s;
  src = 0;
  len = 0;
  if ((int)r < wd * wd && y >= 0 && z >= 0 && y < (int)ng.dims[1] && z < (int)ng.dims[2]) {
    const uint32_t xlo = cx >= (uint32_t)s ? cx - s : 0;
    const uint32_t xhi = cx + s < ng.dims[0] ? cx + s : ng.dims[0] - 1;
    const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
    src = a.nstart[row + xlo];
    len = a.nstart[row + xhi + 1] - src;
  }
}

// Half stencil of cell c for the forward over unordered pairs, run r of (2s+1)s + s + 1: the
// rows above (dz > 0, every dy), the rows ahead in the same plane (dz = 0, dy > 0), both over
// cx-s .. cx+s, and the cells after c in its own row (cx+1 .. cx+s).  With the pairs inside the
// cell (j > i) every unordered pair within the stencil is met once.
__device__ __forceinline__ void soft_half_run(const SoftArgs& a, const Geo& ng, uint32_t c, uint32_t r,
                                              uint32_t& src, uint32_t& len) {
  const int s = a.stencil, wd = 2 * s + 1;
  const uint32_t cx = c % ng.dims[0], cy = (c / ng.dims[0]) % ng.dims[1], cz = c / (ng.dims[0] * ng.dims[1]);
  src = 0;
  len = 0;
  int dy, dz;
  uint32_t xlo = cx >= (uint32_t)s ? cx - s : 0;
  const uint32_t xhi = cx + s < ng.dims[0] ? cx + s : ng.dims[0] - 1;
  if ((int)r < s * wd) {
    dz = 1 + (int)r / wd, dy = (int)r % wd - s;
  } else if ((int)r < s * wd + s) {
    dz = 0, dy = 1 + (int)r - s * wd;
  } else if ((int)r == s * wd + s) {
    dz = 0, dy = 0, xlo = cx + 1;
  } else {
    return;
  }
  const int y = (int)cy + dy, z = (int)cz + dz;
  if (y < 0 || y >= (int)ng.dims[1] || z >= (int)ng.dims[2] || xlo > xhi) return;
  const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
  src = a.nstart[row + xlo];
  len = a.nstart[row + xhi + 1] - src;
}

// Iterates the items of the owner list (the centrals; candidates: their full stencil of
// neighbours, whose staged .w is the ion index so that the owner itself is skipped) with the
// candidates staged 32 at a time as interleaved pairs (xa xb ya yb za zb wa wb) and tested two at
// a time with packed float32 math; the in-range pairs of every half-batch of 16 candidates go to
// a warp list that all lanes then process: hit(d2, 1) for each.  item_hook(cnt, n_cand) runs once
// per item.
template <class H, class I>
__device__ __forceinline__ void soft_items_listed(const SoftArgs& a, float* bf, uint32_t* rsrc, uint32_t* rpre,
                                                  float* wlist, H&& hit, I&& item_hook) {
  const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  const Geo ng = *a.ngeo;
  const uint32_t n_front = a.ogeo->work_n2, n_items = n_front + a.ogeo->work_n3;
  const int s = a.stencil, wd = 2 * s + 1;
  const int n_runs = wd * wd;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&a.ogeo->work_next2, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const uint2 it = work_item(a.oitem, a.ocap, n_front, item);
    const uint32_t c = it.x, first = it.y >> 6, cnt = it.y & 63u;
    const uint32_t c0 = a.ostart[c] + first;
    const uint32_t n_cand = run_table(lane, n_runs, rsrc, rpre, [&](uint32_t r, uint32_t& src, uint32_t& len) {
      soft_run(a, ng, c, r, src, len);
    });
    item_hook(cnt, n_cand);
    const bool valid = lane < cnt;
    float4 p = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float emax = -INFINITY;
    uint32_t pidx = ~0u;
    if (valid) {
      p = a.orec[c0 + lane];
      pidx = __float_as_uint(p.w);
      emax = a.rc2u;
    }
    const unsigned long long px = f2_pack(p.x, p.x), py = f2_pack(p.y, p.y), pz = f2_pack(p.z, p.z);
    int rr = 0;
    auto fetch = [&](uint32_t pos) -> float4 {
      if (pos >= n_cand) return make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(~0u));
      while (pos >= rpre[rr + 1]) ++rr;
      return __ldg(a.nrec + rsrc[rr] + (pos - rpre[rr]));
    };
    float4 nxt = fetch(lane);
    for (uint32_t b = 0; b < n_cand; b += 32) {
      __syncwarp();
      {
        float* d = bf + (lane >> 1) * 8 + (lane & 1);
        d[0] = nxt.x, d[2] = nxt.y, d[4] = nxt.z, d[6] = nxt.w;
      }
      __syncwarp();
      nxt = fetch(b + 32 + lane);
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        uint32_t nh = 0;
#pragma unroll 2
        for (uint32_t u = 0; u < 8; ++u) {
          const uint32_t t = 8 * half + u;
          const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(bf)[2 * t];
          const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(bf)[2 * t + 1];
          float d2a, d2b, wa, wb;
          dist2_x2(px, py, pz, xy.x, xy.y, zw.x, d2a, d2b);
          f2_unpack(zw.y, wa, wb);
          const bool ha = d2a < emax && __float_as_uint(wa) != pidx;
          const bool hb = d2b < emax && __float_as_uint(wb) != pidx;
          const uint32_t ba = __ballot_sync(0xffffffffu, ha);
          wlist[ha ? nh + __popc(ba & lt) : 512 + lane] = d2a;
          nh += __popc(ba);
          const uint32_t bb = __ballot_sync(0xffffffffu, hb);
          wlist[hb ? nh + __popc(bb & lt) : 512 + lane] = d2b;
          nh += __popc(bb);
        }
        __syncwarp();
        for (uint32_t h = lane; h < nh; h += 32) hit(wlist[h], 1.f);
        __syncwarp();
      }
    }
  }
}

// The forward over unordered pairs, cell by cell: a warp takes a share of the cells left (at
// most 32, at least 1, from the counter a.ogeo->work_next2) and, for each non-empty cell, tests
// the half stencil's records (the lanes, 32 per load, each in registers) against the cell's
// records (staged in shared memory up to 64 at a time as interleaved pairs xa xb ya yb za zb ea
// eb and read by every lane at once, two per packed test), so that the lanes stay busy whatever
// the cell's record count; the pairs inside the cell (j > i) are tested by each lane on its own.
// A record's e (and a candidate's) is rc^2 for a central and -1 otherwise: a pair is in range
// below max(e_rec, e_cand), weight 2 (the sign bit of its listed d2) when both are central.
// hit(d2, weight) per in-range pair; cell_hook(m, n_cand) once per cell before its pairs.
template <class H, class C>
__device__ __forceinline__ void soft_cells_sym(const SoftArgs& a, float* gf, uint32_t* rsrc, uint32_t* rpre,
                                               uint32_t* wlist, H&& hit, C&& cell_hook) {
  const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  const Geo ng = *a.ngeo;
  const uint32_t n_cells = ng.n_cells;
  const int s = a.stencil, n_runs = s * (2 * s + 1) + s + 1;
  const float E = a.rc2u;
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  for (;;) {
    uint32_t base = 0, take = 0;
    if (lane == 0) {
      const uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&a.ogeo->work_next2);
      const uint32_t left = cur < n_cells ? n_cells - cur : 0u;
      take = min(32u, max(1u, left / (8 * n_warps)));
      base = atomicAdd(&a.ogeo->work_next2, take);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    take = __shfl_sync(0xffffffffu, take, 0);
    if (base >= n_cells) break;
    uint32_t s0 = 0, s1 = 0;
    if (lane < take && base + lane < n_cells) s0 = a.ostart[base + lane], s1 = a.ostart[base + lane + 1];
    uint32_t todo = __ballot_sync(0xffffffffu, s1 > s0);
    while (todo) {
      const int src_lane = __ffs(todo) - 1;
      todo &= todo - 1u;
      const uint32_t c = base + (uint32_t)src_lane;
      const uint32_t a0 = __shfl_sync(0xffffffffu, s0, src_lane), a1 = __shfl_sync(0xffffffffu, s1, src_lane);
      const uint32_t n_cand = run_table(lane, n_runs, rsrc, rpre, [&](uint32_t r, uint32_t& src, uint32_t& len) {
        soft_half_run(a, ng, c, r, src, len);
      });
      cell_hook(a1 - a0, n_cand + (a1 - a0));
      // pairs inside the cell
      for (uint32_t i0 = a0; i0 < a1; i0 += 32) {
        const uint32_t i = i0 + lane;
        if (i < a1) {
          const float4 p = __ldg(a.orec + i);
          const float ci = (float)(__ldg(a.pfx + i + 1) - __ldg(a.pfx + i));
          for (uint32_t j = i + 1; j < a1; ++j) {
            const float4 q = __ldg(a.orec + j);
            const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
            const float wt = ci + (float)(__ldg(a.pfx + j + 1) - __ldg(a.pfx + j));
            if (d2 < E && wt > 0.f) hit(d2, wt);
          }
        }
      }
      if (n_cand == 0) continue;
      for (uint32_t g0 = a0; g0 < a1; g0 += 64) {
        const uint32_t m = min(64u, a1 - g0), n_pr = (m + 1) >> 1;
        __syncwarp();
#pragma unroll
        for (uint32_t h = 0; h < 64; h += 32) {
          const uint32_t r = h + lane;
          if (r < 2 * n_pr) {
            float4 q = make_float4(INFINITY, INFINITY, INFINITY, -1.f);  // the pad of an odd group never hits
            if (r < m) {
              q = __ldg(a.orec + g0 + r);
              q.w = __ldg(a.pfx + g0 + r + 1) > __ldg(a.pfx + g0 + r) ? E : -1.f;
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
          q.w = __ldg(a.pfx + j + 1) > __ldg(a.pfx + j) ? E : -1.f;
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
            uint32_t nh = 0;
#pragma unroll 4
            for (uint32_t k = k0; k < k1; ++k) {
              const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(gf)[2 * k];
              const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(gf)[2 * k + 1];
              float d2a, d2b, ea, eb;
              dist2_x2(xy.x, xy.y, zw.x, qx, qy, qz, d2a, d2b);
              f2_unpack(zw.y, ea, eb);
              const bool ha = d2a < fmaxf(eq, ea), hb = d2b < fmaxf(eq, eb);
              const uint32_t va = __float_as_uint(d2a) | (~__float_as_uint(ea) & w2q);
              const uint32_t vb = __float_as_uint(d2b) | (~__float_as_uint(eb) & w2q);
              const uint32_t ba = __ballot_sync(0xffffffffu, ha);
              wlist[ha ? nh + __popc(ba & lt) : 512 + lane] = va;
              nh += __popc(ba);
              const uint32_t bb = __ballot_sync(0xffffffffu, hb);
              wlist[hb ? nh + __popc(bb & lt) : 512 + lane] = vb;
              nh += __popc(bb);
            }
            __syncwarp();
            for (uint32_t h = lane; h < nh; h += 32) {
              const uint32_t v = wlist[h];
              hit(__uint_as_float(v & 0x7FFFFFFFu), (v >> 31) ? 2.f : 1.f);
            }
            __syncwarp();
          }
        }
      }
    }
  }
}

// Same iteration for the adjoint, where every in-range pair updates its owner lane's
// accumulators: f(p, qx, qy, qz, qw, d2) under a branch per candidate (queueing the pairs
// first measured slower).  ONE: owners and candidates are the neighbour records and the staged
// .w is the candidate's central flag (from the central prefix); a pair counts when d2 > 0 and
// either end is central.  Otherwise .w is the ion index and the owner itself is skipped.
// begin_owner(valid, p, c_own) / end_owner(valid, p) bracket each owner.
template <bool ONE, class F, class B, class E>
__device__ __forceinline__ void soft_items_owned(const SoftArgs& a, float* bf, uint32_t* rsrc, uint32_t* rpre,
                                                 F&& f, B&& begin_owner, E&& end_owner) {
  const uint32_t lane = threadIdx.x & 31;
  const Geo ng = *a.ngeo;
  const uint32_t n_front = a.ogeo->work_n2, n_items = n_front + a.ogeo->work_n3;
  const int n_runs = (2 * a.stencil + 1) * (2 * a.stencil + 1);
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&a.ogeo->work_next2, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const uint2 it = work_item(a.oitem, a.ocap, n_front, item);
    const uint32_t c = it.x, first = it.y >> 6, cnt = it.y & 63u;
    const uint32_t c0 = a.ostart[c] + first;
    const uint32_t n_cand = run_table(lane, n_runs, rsrc, rpre, [&](uint32_t r, uint32_t& src, uint32_t& len) {
      soft_run(a, ng, c, r, src, len);
    });
    const bool valid = lane < cnt;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    float c_own = 0.f;
    if (valid) {
      p = a.orec[c0 + lane];
      if (ONE) c_own = (float)(__ldg(a.pfx + c0 + lane + 1) - __ldg(a.pfx + c0 + lane));
    }
    const uint32_t pidx = valid ? __float_as_uint(p.w) : ~0u;
    const float emax = valid ? a.rc2u : -INFINITY;
    const unsigned long long px = f2_pack(p.x, p.x), py = f2_pack(p.y, p.y), pz = f2_pack(p.z, p.z);
    begin_owner(valid, p, c_own);
    int rr = 0;
    auto fetch = [&](uint32_t pos) -> float4 {
      if (pos >= n_cand) return make_float4(INFINITY, INFINITY, INFINITY, ONE ? 0.f : __uint_as_float(~0u));
      while (pos >= rpre[rr + 1]) ++rr;
      const uint32_t j = rsrc[rr] + (pos - rpre[rr]);
      float4 q = __ldg(a.nrec + j);
      if (ONE) q.w = (float)(__ldg(a.pfx + j + 1) - __ldg(a.pfx + j));
      return q;
    };
    auto hit = [&](float d2, float w) -> bool {
      if (ONE) return d2 < emax && d2 > 0.f && c_own + w > 0.f;
      return d2 < emax && __float_as_uint(w) != pidx;
    };
    float4 nxt = fetch(lane);
    for (uint32_t b = 0; b < n_cand; b += 32) {
      __syncwarp();
      {
        float* d = bf + (lane >> 1) * 8 + (lane & 1);
        d[0] = nxt.x, d[2] = nxt.y, d[4] = nxt.z, d[6] = nxt.w;
      }
      __syncwarp();
      nxt = fetch(b + 32 + lane);
#pragma unroll 2
      for (uint32_t t = 0; t < 16; ++t) {
        const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(bf)[2 * t];
        const ulonglong2 zw = reinterpret_cast<const ulonglong2*>(bf)[2 * t + 1];
        float d2a, d2b, xa, xb, ya, yb, za, zb, wa, wb;
        dist2_x2(px, py, pz, xy.x, xy.y, zw.x, d2a, d2b);
        f2_unpack(zw.y, wa, wb);
        if (hit(d2a, wa)) {
          f2_unpack(xy.x, xa, xb), f2_unpack(xy.y, ya, yb), f2_unpack(zw.x, za, zb);
          f(p, xa, ya, za, wa, d2a);
        }
        if (hit(d2b, wb)) {
          f2_unpack(xy.x, xa, xb), f2_unpack(xy.y, ya, yb), f2_unpack(zw.x, za, zb);
          f(p, xb, yb, zb, wb, d2b);
        }
      }
    }
    end_owner(valid, p);
  }
}

// ---------------------------------------------------------------------------
// forward: fine-grid moments
// ---------------------------------------------------------------------------
template <bool SYM>
__global__ void __launch_bounds__(256) k_soft_fwd(const SoftArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_grp[8][64];        // per warp: staged records (the cell's, or a batch of candidates)
  __shared__ float s_hits[8][512 + 32];  // per warp: one half-batch's in-range d2 + a trash row
  __shared__ uint32_t s_rsrc[8][kSoftRuns], s_rpre[8][kSoftRuns + 1];
  // 32-bit counts per CTA; a warp whose item could push the CTA past 2^31 (weighted) pairs writes
  // to global instead
  uint32_t* sM0 = reinterpret_cast<uint32_t*>(smem);
  float* sM1 = reinterpret_cast<float*>(smem + a.n_fine * 4);
  float* sM2 = reinterpret_cast<float*>(smem + a.n_fine * 8);
  __shared__ unsigned long long s_pairs;
  for (uint32_t m = threadIdx.x; m < a.n_fine; m += blockDim.x) sM0[m] = 0, sM1[m] = 0.f, sM2[m] = 0.f;
  if (threadIdx.x == 0) s_pairs = 0;
  __syncthreads();
  bool glob = false;
  const uint32_t w = threadIdx.x >> 5;
  const float s = a.scale, inv_w = a.inv_w, wf = a.w, rc = a.rc;
  const uint32_t nf = a.n_fine;
  // one pair at distance sqrt(d2) with weight wt (1 or 2) into the fine-grid moments
  auto pair = [&](float d2, float wt) {
    const float u = s * (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f);
    if (!(u < rc)) return;
    uint32_t m = (uint32_t)(u * inv_w);
    m = m < nf ? m : nf - 1;
    const float delta = u - ((float)m + 0.5f) * wf;
    const float wd = wt * delta;
    if (glob) {
      atomicAdd(&a.M0[m], (unsigned long long)wt);
      atomicAdd(&a.M1[m], (double)wd);
      atomicAdd(&a.M2[m], (double)wd * (double)delta);
    } else {
      atomicAdd(&sM0[m], (uint32_t)wt);
      atomicAdd(&sM1[m], wd);
      atomicAdd(&sM2[m], wd * delta);
    }
  };
  auto bound = [&](uint32_t cnt, uint32_t n_cand) {
    unsigned long long old = 0;
    const unsigned long long inc = (unsigned long long)cnt * n_cand * (SYM ? 2u : 1u);
    if ((threadIdx.x & 31) == 0) old = atomicAdd(&s_pairs, inc);
    old = __shfl_sync(0xffffffffu, old, 0);
    glob = old + inc >= (1ull << 31);
  };
  if (SYM)
    soft_cells_sym(a, reinterpret_cast<float*>(s_grp[w]), s_rsrc[w], s_rpre[w], reinterpret_cast<uint32_t*>(s_hits[w]),
                   pair, bound);
  else
    soft_items_listed(a, reinterpret_cast<float*>(s_grp[w]), s_rsrc[w], s_rpre[w], s_hits[w], pair, bound);
  __syncthreads();
  for (uint32_t m = threadIdx.x; m < nf; m += blockDim.x) {
    if (sM0[m]) {
      atomicAdd(&a.M0[m], (unsigned long long)sM0[m]);
      atomicAdd(&a.M1[m], (double)sM1[m]);
      atomicAdd(&a.M2[m], (double)sM2[m]);
    }
  }
}

// d^n/du^n of Phi((e - u)/sigma), n = 0..3, in FP64
__device__ __forceinline__ void phi_derivs(double e, double u, double sigma, double out[4]) {
  const double t = (e - u) / sigma;
  const double ph = exp(-0.5 * t * t) * 0.39894228040143267794;  // 1/sqrt(2 pi)
  out[0] = 0.5 * erfc(-t * 0.70710678118654752440);
  out[1] = -ph / sigma;
  out[2] = -t * ph / (sigma * sigma);
  out[3] = (1.0 - t * t) * ph / (sigma * sigma * sigma);
}

// h[b] = sum_m M0 K_b + M1 K_b' + M2/2 K_b'' (one block per bin)
__global__ void __launch_bounds__(256) k_soft_finalize(const unsigned long long* __restrict__ M0,
                                                       const double* __restrict__ M1, const double* __restrict__ M2,
                                                       uint32_t n_fine, double w, double r0, double dr, double sigma,
                                                       float* __restrict__ h) {
  griddep_wait();
  griddep_launch();
  __shared__ double s_part[8];
  const uint32_t b = blockIdx.x;
  const double e0 = r0 + (double)b * dr, e1 = r0 + (double)(b + 1) * dr;
  double acc = 0.0;
  for (uint32_t m = threadIdx.x; m < n_fine; m += blockDim.x) {
    const unsigned long long n0 = M0[m];
    if (!n0) continue;
    const double c = ((double)m + 0.5) * w;
    double p1[4], p0[4];
    phi_derivs(e1, c, sigma, p1);
    phi_derivs(e0, c, sigma, p0);
    acc += (double)n0 * (p1[0] - p0[0]) + M1[m] * (p1[1] - p0[1]) + 0.5 * M2[m] * (p1[2] - p0[2]);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_part[i];
    h[b] = (float)t;
  }
}

// T[0][m] = W(c_m), T[1][m] = W'(c_m), T[2][m] = W''(c_m) for W(u) = sum_b G[b] K_b'(u)
__global__ void __launch_bounds__(256) k_soft_table(const float* __restrict__ G, uint32_t n_bins, uint32_t n_fine,
                                                    double w, double r0, double dr, double sigma,
                                                    float* __restrict__ T) {
  griddep_wait();
  griddep_launch();
  const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_fine) return;
  const double c = ((double)m + 0.5) * w;
  double a1 = 0.0, a2 = 0.0, a3 = 0.0;
  double pl[4];
  phi_derivs(r0, c, sigma, pl);
  for (uint32_t b = 0; b < n_bins; ++b) {
    double ph[4];
    phi_derivs(r0 + (double)(b + 1) * dr, c, sigma, ph);
    const double g = (double)G[b];
    a1 += g * (ph[1] - pl[1]);
    a2 += g * (ph[2] - pl[2]);
    a3 += g * (ph[3] - pl[3]);
    for (int k = 0; k < 4; ++k) pl[k] = ph[k];
  }
  T[m] = (float)a1;
  T[n_fine + m] = (float)a2;
  T[2 * n_fine + m] = (float)a3;
}

// ---------------------------------------------------------------------------
// adjoint passes
// ---------------------------------------------------------------------------
// ONE: a single pass over the neighbour records when the centrals are among them; every record
// owns its gradient, W s (x_o - x_c)/d times the pair's weight (central flags of both ends
// added), and the central owners accumulate dL/ds.  Otherwise pass A (owners = centrals, write)
// and pass B (owners = neighbours, add).
template <bool ONE>
__global__ void __launch_bounds__(256) k_soft_bwd(const SoftArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_buf[8][32];
  __shared__ uint32_t s_rsrc[8][kSoftRuns], s_rpre[8][kSoftRuns + 1];
  __shared__ double s_gs[8];
  float* sT = reinterpret_cast<float*>(smem);
  for (uint32_t m = threadIdx.x; m < 3 * a.n_fine; m += blockDim.x) sT[m] = a.T[m];
  __syncthreads();
  const uint32_t w = threadIdx.x >> 5;
  const float s = a.scale, inv_w = a.inv_w, wf = a.w, rc = a.rc;
  const uint32_t nf = a.n_fine;
  float gx = 0.f, gy = 0.f, gz = 0.f, c_self = 0.f;
  double gs_lane = 0.0;
  float gs_item = 0.f;
  auto begin = [&](bool, const float4&, float c_own) { gx = gy = gz = 0.f, gs_item = 0.f, c_self = c_own; };
  auto pair = [&](const float4& p, float qx, float qy, float qz, float qw, float d2) {
    const float rs = d2 > 0.f ? rsqrtf(d2) : 0.f;
    const float d = d2 * rs;
    const float u = s * d;
    if (!(u < rc)) return;
    uint32_t m = (uint32_t)(u * inv_w);
    m = m < nf ? m : nf - 1;
    const float delta = u - ((float)m + 0.5f) * wf;
    const float W = sT[m] + delta * (sT[nf + m] + 0.5f * delta * sT[2 * nf + m]);
    const float f = W * s * rs * (ONE ? c_self + qw : 1.f);  // W s / d (0 for coincident ions), weighted
    gx += f * (p.x - qx);
    gy += f * (p.y - qy);
    gz += f * (p.z - qz);
    if (!ONE || c_self > 0.f) gs_item += W * d;
  };
  auto end = [&](bool valid, const float4& p) {
    if (!valid) return;
    const uint32_t idx = __float_as_uint(p.w);
    float* g = a.grad + 3 * (int64_t)idx;
    if (!ONE && a.pass_b) {
      // owners are neighbours j: dL/dx_j = -sum W s (x_i - x_j)/d, here p = x_j, q = x_i
      g[0] += gx, g[1] += gy, g[2] += gz;
    } else {
      g[0] = gx, g[1] = gy, g[2] = gz;
      gs_lane += (double)gs_item;
    }
  };
  soft_items_owned<ONE>(a, reinterpret_cast<float*>(s_buf[w]), s_rsrc[w], s_rpre[w], pair, begin, end);
  if (ONE || !a.pass_b) {
    for (int o = 16; o > 0; o >>= 1) gs_lane += __shfl_xor_sync(0xffffffffu, gs_lane, o);
    if ((threadIdx.x & 31) == 0) s_gs[w] = gs_lane;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_gs[i];
      atomicAdd(a.grad_s, t);
    }
  }
}

// warp items (cell, first << 6 | count) over every non-empty cell of a list
__global__ void __launch_bounds__(256) k_make_items(const uint32_t* __restrict__ count, Geo* geo,
                                                    uint2* __restrict__ item) {
  griddep_wait();
  griddep_launch();
  const uint32_t nc = geo->n_cells;
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t base = blockIdx.x * blockDim.x; base < nc; base += gridDim.x * blockDim.x) {
    const uint32_t c = base + threadIdx.x;
    const uint32_t v = c < nc ? count[c] : 0u;
    const uint32_t m = v == 0 ? 0u : (v + 31u) / 32u;
    uint32_t x = m;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    uint32_t b0 = 0;
    if (lane == 31 && total) b0 = atomicAdd(&geo->work_n2, total);
    b0 = __shfl_sync(0xffffffffu, b0, 31);
    uint32_t slot = b0 + x - m;
    if (m) {
      const uint32_t bs = v / m, rem = v % m;
      uint32_t first = 0;
      for (uint32_t q = 0; q < m; ++q) {
        const uint32_t cnt = bs + (q < rem ? 1u : 0u);
        item[slot++] = make_uint2(c, (first << 6) | cnt);
        first += cnt;
      }
    }
  }
}

__global__ void k_reset_items(Geo* geo) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) geo->work_n2 = 0, geo->work_n3 = 0, geo->work_next2 = 0;
}

__global__ void k_reset_counter(Geo* geo) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) geo->work_next2 = 0;
}

__global__ void k_soft_gs_out(const double* __restrict__ gs, float* __restrict__ out) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) *out = (float)*gs;
}

static int soft_setup(ps_grid* g, float sigma, float scale, ps_bins bins, SoftArgs& sa, double& w_out) {
  if (!(sigma > 0.0f) || !std::isfinite(sigma)) return fail(PS_ERR_INVALID_ARG, "smoothed RDF: sigma must be > 0");
  if (!(scale > 0.0f) || !std::isfinite(scale)) return fail(PS_ERR_INVALID_ARG, "smoothed RDF: scale must be > 0");
  const double stop = bins.r0 + (double)bins.n_bins * bins.dr;
  const double rc = stop + 6.0 * (double)sigma;
  if ((double)g->r_cut * (double)scale < rc * (1.0 + 1e-6))
    return fail(PS_ERR_INVALID_ARG, "smoothed RDF: grid r_cut * scale must cover stop + 6 sigma");
  double w = (double)sigma / 40.0;
  if (rc / w > (double)kSoftFineMax) w = rc / (double)kSoftFineMax;
  sa.n_fine = (uint32_t)std::ceil(rc / w);
  if (sa.n_fine > kSoftFineMax) sa.n_fine = kSoftFineMax;
  sa.w = (float)w;
  sa.inv_w = (float)(1.0 / w);
  sa.scale = scale;
  sa.sigma = sigma;
  sa.rc = (float)rc;
  const double rcu = rc / (double)scale;
  sa.rc2u = (float)(rcu * rcu * (1.0 + 1e-6));
  sa.stencil = g->stencil;
  w_out = w;
  return PS_OK;
}

static int launch_grid_for(const ps_grid* g, const void* kern, uint32_t smem, int* blocks) {
  int per_sm = 0;
  PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
  if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "smoothed RDF kernel does not fit on an SM");
  *blocks = g->num_sms * per_sm;
  return PS_OK;
}

// The centrals are neighbour records (the central list then carries the central prefix over the
// neighbour records, g->cr).
static bool centrals_in_neighbours(const ps_grid* g, const uint64_t ctr_mask[4]) {
  bool subset = !g->pack_type;
  for (int w = 0; w < 4; ++w) subset = subset && (ctr_mask[w] & ~g->nbr_mask[w]) == 0;
  return subset;
}

// Owners = the neighbour records: warp items over the non-empty neighbour cells.
static int nbr_items(ps_grid* g, SoftArgs& sa, cudaStream_t s, uint32_t kid) {
  PS_LAUNCH(kid, s, PS_CUDA(launch_pdl(k_reset_items, 1, 32, 0, s, g->nbr.geo)));
  PS_LAUNCH(kid, s, PS_CUDA(launch_pdl(k_make_items, g->num_sms * 4, 256, 0, s, g->nbr.count, g->nbr.geo, g->nbr_witem)));
  sa.orec = g->nbr.rec;
  sa.ostart = g->nbr.start;
  sa.oitem = g->nbr_witem;
  sa.ocap = g->item_cap;
  sa.ogeo = g->nbr.geo;
  return PS_OK;
}

int soft_forward(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma, float scale,
                 ps_bins bins, float* d_h, cudaStream_t s) {
  SoftArgs sa;
  memset(&sa, 0, sizeof(sa));
  double w = 0.0;
  int rc = soft_setup(g, sigma, scale, bins, sa, w);
  if (rc) return rc;
  ZeroOut z;  // the moment accumulators are zeroed by the central-list reset kernel
  z.p[0] = reinterpret_cast<uint64_t*>(g->soft_m0);
  z.p[1] = reinterpret_cast<uint64_t*>(g->soft_m1);
  z.p[2] = reinterpret_cast<uint64_t*>(g->soft_m2);
  z.n[0] = z.n[1] = z.n[2] = sa.n_fine;
  rc = build_central_list(g, dsrf, ctr_mask, dsrf_min, s, z);
  if (rc) return rc;
  sa.nrec = g->nbr.rec;
  sa.nstart = g->nbr.start;
  sa.ngeo = g->nbr.geo;
  sa.M0 = g->soft_m0;
  sa.M1 = g->soft_m1;
  sa.M2 = g->soft_m2;
  const uint32_t smem = sa.n_fine * 12;
  int blocks = 0;
  if (centrals_in_neighbours(g, ctr_mask)) {
    // unordered pairs of neighbour records, weighted by the central flags of both ends
    rc = launch_grid_for(g, (const void*)k_soft_fwd<true>, smem, &blocks);
    if (rc) return rc;
    // cells taken from the neighbour list's counter (owners = candidates = neighbour records)
    PS_LAUNCH(PS_KID_SOFT_FWD, s, PS_CUDA(launch_pdl(k_reset_items, 1, 32, 0, s, g->nbr.geo)));
    sa.orec = g->nbr.rec;
    sa.ostart = g->nbr.start;
    sa.ogeo = g->nbr.geo;
    sa.pfx = reinterpret_cast<const uint32_t*>(g->cr);
    PS_LAUNCH(PS_KID_SOFT_FWD, s, PS_CUDA(launch_pdl(k_soft_fwd<true>, blocks, 256, smem, s, sa)));
  } else {
    rc = launch_grid_for(g, (const void*)k_soft_fwd<false>, smem, &blocks);
    if (rc) return rc;
    sa.orec = g->ctr.rec;
    sa.ostart = g->ctr.start;
    sa.oitem = g->ctr.witem;
    sa.ocap = g->item_cap;
    sa.ogeo = g->ctr.geo;
    PS_LAUNCH(PS_KID_SOFT_FWD, s, PS_CUDA(launch_pdl(k_soft_fwd<false>, blocks, 256, smem, s, sa)));
  }
  PS_LAUNCH(PS_KID_SOFT_FWD, s,
            PS_CUDA(launch_pdl(k_soft_finalize, bins.n_bins, 256, 0, s, g->soft_m0, g->soft_m1, g->soft_m2, sa.n_fine, w, bins.r0,
                                                        bins.dr, (double)sigma, d_h)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int soft_backward(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma, float scale,
                  ps_bins bins, const float* d_G, float* d_grad, float* d_grad_s, cudaStream_t s) {
  SoftArgs sa;
  memset(&sa, 0, sizeof(sa));
  double w = 0.0;
  int rc = soft_setup(g, sigma, scale, bins, sa, w);
  if (rc) return rc;
  rc = build_central_list(g, dsrf, ctr_mask, dsrf_min, s);
  if (rc) return rc;
  PS_CUDA(cudaMemsetAsync(d_grad, 0, (size_t)g->n * 3 * sizeof(float), s));
  PS_CUDA(cudaMemsetAsync(g->soft_gs, 0, sizeof(double), s));
  PS_LAUNCH(PS_KID_SOFT_BWD, s,
            PS_CUDA(launch_pdl(k_soft_table, (sa.n_fine + 255) / 256, 256, 0, s, d_G, bins.n_bins, sa.n_fine, w, bins.r0, bins.dr,
                                                                 (double)sigma, g->soft_T)));
  sa.T = g->soft_T;
  sa.grad = d_grad;
  sa.grad_s = g->soft_gs;
  const uint32_t smem = sa.n_fine * 12;
  int blocks = 0;
  if (centrals_in_neighbours(g, ctr_mask)) {
    // one pass: the central prefix over the neighbour records (built with the central list) gives
    // every record's central flag
    rc = launch_grid_for(g, (const void*)k_soft_bwd<true>, smem, &blocks);
    if (rc) return rc;
    rc = nbr_items(g, sa, s, PS_KID_SOFT_BWD);
    if (rc) return rc;
    sa.nrec = g->nbr.rec;
    sa.nstart = g->nbr.start;
    sa.ngeo = g->nbr.geo;
    sa.pfx = reinterpret_cast<const uint32_t*>(g->cr);
    PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_bwd<true>, blocks, 256, smem, s, sa)));
  } else {
    rc = launch_grid_for(g, (const void*)k_soft_bwd<false>, smem, &blocks);
    if (rc) return rc;
    // pass A: owners = centrals, candidates = neighbours
    sa.orec = g->ctr.rec;
    sa.ostart = g->ctr.start;
    sa.oitem = g->ctr.witem;
    sa.ocap = g->item_cap;
    sa.ogeo = g->ctr.geo;
    sa.nrec = g->nbr.rec;
    sa.nstart = g->nbr.start;
    sa.ngeo = g->nbr.geo;
    sa.pass_b = 0;
    PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_bwd<false>, blocks, 256, smem, s, sa)));
    // pass B: owners = neighbours, candidates = centrals
    rc = nbr_items(g, sa, s, PS_KID_SOFT_BWD);
    if (rc) return rc;
    sa.nrec = g->ctr.rec;
    sa.nstart = g->ctr.start;
    sa.ngeo = g->nbr.geo;
    sa.pass_b = 1;
    PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_bwd<false>, blocks, 256, smem, s, sa)));
  }
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_gs_out, 1, 32, 0, s, g->soft_gs, d_grad_s)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
