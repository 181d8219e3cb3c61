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
// recomputed, never stored.  Pass A (one lane per central i) writes dL/dx_i and
// accumulates dL/ds; pass B (one lane per neighbour j, candidates = centrals)
// adds dL/dx_j.  Each gradient has one owner: no atomics on the gradient.
#include <cmath>
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

constexpr int kSoftRuns = 25;

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

// Iterates the items of the owner list; for every owner lane and in-range
// candidate calls f(lane_has_owner, p (owner record), q (candidate), d2).
struct NoHook {
  __device__ void operator()(uint32_t, uint32_t) const {}
};

template <class F, class B, class E, class H = NoHook>
__device__ __forceinline__ void soft_items(const SoftArgs& a, float4* buf, uint32_t* rsrc, uint32_t* rpre, F&& f,
                                           B&& begin_owner, E&& end_owner, H&& item_hook = H()) {
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
    uint32_t src = 0, len = 0;
    soft_run(a, ng, c, lane, src, len);
    uint32_t pre = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= (uint32_t)o) pre += y;
    }
    const uint32_t n_cand = __shfl_sync(0xffffffffu, pre, 31);
    __syncwarp();
    if (lane < (uint32_t)n_runs) {
      rsrc[lane] = src;
      rpre[lane + 1] = pre;
    }
    if (lane == 0) rpre[0] = 0;
    __syncwarp();
    item_hook(cnt, n_cand);
    const bool valid = lane < cnt;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) p = a.orec[c0 + lane];
    begin_owner(valid, p);
    int rr = 0;
    auto fetch = [&](uint32_t pos) -> float4 {
      if (pos >= n_cand) return make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(~0u));
      while (pos >= rpre[rr + 1]) ++rr;
      return __ldg(a.nrec + rsrc[rr] + (pos - rpre[rr]));
    };
    float4 nxt = fetch(lane);
    for (uint32_t b = 0; b < n_cand; b += 32) {
      __syncwarp();
      buf[lane] = nxt;
      __syncwarp();
      nxt = fetch(b + 32 + lane);
      if (valid) {
#pragma unroll 4
        for (int t = 0; t < 32; ++t) {
          const float4 q = buf[t];
          const float d2 = dist2(p.x, p.y, p.z, q.x, q.y, q.z);
          if (d2 < a.rc2u && __float_as_uint(q.w) != __float_as_uint(p.w)) f(p, q, d2);
        }
      }
    }
    end_owner(valid, p);
  }
}

// ---------------------------------------------------------------------------
// forward: fine-grid moments
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_soft_fwd(const SoftArgs a) {
  griddep_wait();
  griddep_launch();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float4 s_buf[8][32];
  __shared__ uint32_t s_rsrc[8][kSoftRuns], s_rpre[8][kSoftRuns + 1];
  // 32-bit counts per CTA; a warp whose item could push the CTA past 2^31 pairs writes to global instead
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
  auto pair = [&](const float4& p, const float4& q, float d2) {
    const float u = s * (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f);
    if (!(u < rc)) return;
    uint32_t m = (uint32_t)(u * inv_w);
    m = m < nf ? m : nf - 1;
    const float delta = u - ((float)m + 0.5f) * wf;
    if (glob) {
      atomicAdd(&a.M0[m], 1ull);
      atomicAdd(&a.M1[m], (double)delta);
      atomicAdd(&a.M2[m], (double)delta * (double)delta);
    } else {
      atomicAdd(&sM0[m], 1u);
      atomicAdd(&sM1[m], delta);
      atomicAdd(&sM2[m], delta * delta);
    }
  };
  auto bound = [&](uint32_t cnt, uint32_t n_cand) {
    unsigned long long old = 0;
    const unsigned long long inc = (unsigned long long)cnt * n_cand;
    if ((threadIdx.x & 31) == 0) old = atomicAdd(&s_pairs, inc);
    old = __shfl_sync(0xffffffffu, old, 0);
    glob = old + inc >= (1ull << 31);
  };
  auto nop = [](bool, const float4&) {};
  soft_items(a, s_buf[w], s_rsrc[w], s_rpre[w], pair, nop, nop, bound);
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
  float gx = 0.f, gy = 0.f, gz = 0.f;
  double gs_lane = 0.0;
  float gs_item = 0.f;
  auto begin = [&](bool, const float4&) { gx = gy = gz = 0.f, gs_item = 0.f; };
  auto pair = [&](const float4& p, const float4& q, float d2) {
    const float rs = d2 > 0.f ? rsqrtf(d2) : 0.f;
    const float d = d2 * rs;
    const float u = s * d;
    if (!(u < rc)) return;
    uint32_t m = (uint32_t)(u * inv_w);
    m = m < nf ? m : nf - 1;
    const float delta = u - ((float)m + 0.5f) * wf;
    const float W = sT[m] + delta * (sT[nf + m] + 0.5f * delta * sT[2 * nf + m]);
    const float f = W * s * rs;  // W s / d (0 for coincident ions)
    gx += f * (p.x - q.x);
    gy += f * (p.y - q.y);
    gz += f * (p.z - q.z);
    gs_item += W * d;
  };
  auto end = [&](bool valid, const float4& p) {
    if (!valid) return;
    const uint32_t idx = __float_as_uint(p.w);
    float* g = a.grad + 3 * (int64_t)idx;
    if (a.pass_b) {
      // owners are neighbours j: dL/dx_j = -sum W s (x_i - x_j)/d, here p = x_j, q = x_i
      g[0] += gx, g[1] += gy, g[2] += gz;
    } else {
      g[0] = gx, g[1] = gy, g[2] = gz;
      gs_lane += (double)gs_item;
    }
  };
  soft_items(a, s_buf[w], s_rsrc[w], s_rpre[w], pair, begin, end);
  if (!a.pass_b) {
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
  sa.orec = g->ctr.rec;
  sa.ostart = g->ctr.start;
  sa.oitem = g->ctr.witem;
  sa.ocap = g->item_cap;
  sa.ogeo = g->ctr.geo;
  sa.nrec = g->nbr.rec;
  sa.nstart = g->nbr.start;
  sa.ngeo = g->nbr.geo;
  sa.M0 = g->soft_m0;
  sa.M1 = g->soft_m1;
  sa.M2 = g->soft_m2;
  const uint32_t smem = sa.n_fine * 12;
  int blocks = 0;
  rc = launch_grid_for(g, (const void*)k_soft_fwd, smem, &blocks);
  if (rc) return rc;
  PS_LAUNCH(PS_KID_SOFT_FWD, s, PS_CUDA(launch_pdl(k_soft_fwd, blocks, 256, smem, s, sa)));
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
  rc = launch_grid_for(g, (const void*)k_soft_bwd, smem, &blocks);
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
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_bwd, blocks, 256, smem, s, sa)));
  // pass B: owners = neighbours, candidates = centrals
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_reset_items, 1, 32, 0, s, g->nbr.geo)));
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_make_items, g->num_sms * 4, 256, 0, s, g->nbr.count, g->nbr.geo, g->nbr_witem)));
  sa.orec = g->nbr.rec;
  sa.ostart = g->nbr.start;
  sa.oitem = g->nbr_witem;
  sa.ocap = g->item_cap;
  sa.ogeo = g->nbr.geo;
  sa.nrec = g->ctr.rec;
  sa.nstart = g->ctr.start;
  sa.ngeo = g->nbr.geo;
  sa.pass_b = 1;
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_bwd, blocks, 256, smem, s, sa)));
  PS_LAUNCH(PS_KID_SOFT_BWD, s, PS_CUDA(launch_pdl(k_soft_gs_out, 1, 32, 0, s, g->soft_gs, d_grad_s)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
