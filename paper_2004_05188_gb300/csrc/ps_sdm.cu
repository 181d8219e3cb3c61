// Spatial distribution map: the three-dimensional two-point statistic of which
// the RDF and the kNN distributions are annular integrals (Methods,
// "Descriptive, two-point spatial statistics, and clustering").  For every
// central ion and every neighbour within the ROI radius R (d2 < (float)(R*R)),
// the float32 displacement x_j - x_i is binned into cubic voxels of edge w;
// the paper's setting is w = 0.025 nm with R = 2 nm (Results, strong scaling).
//
// The enumeration is the exact query's: the same cell grid and central list.
// Each central gets one thread; the centrals of a dense cell's item share the
// candidate walk, so their loads of a record broadcast from L1 (cells with at
// most 3 centrals let the lanes split each central's candidates instead);
// sparse cells' items are taken 32 at a time.  Voxel edges V[m] = (float)((m - n_vox/2) * w)
// (double arithmetic) sit in shared memory; a voxel index is guessed from
// (d - V[0]) / w and checked against the table, so the half-open rule
// V[m] <= d < V[m+1] holds exactly.  The map (n_vox^3 uint64 counters, 33 MB
// for the paper's 160^3 voxels) stays L2-resident and takes global atomics.
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

struct SdmArgs {
  const float4* nrec;
  const uint32_t* nstart;
  const Geo* ngeo;
  const float4* crec;
  const uint32_t* cstart;
  const uint32_t* cwork;
  const uint2* witem;
  uint32_t work_cap;
  Geo* cgeo;
  int stencil;
  float ER;  // (float)(R * R)
  double w;
  uint32_t n_vox;
  unsigned long long* H;
  uint64_t* meta;
};

constexpr uint32_t kSdmMaxVox = 1024;
constexpr uint32_t kSdmLightCap = 32 * (kHeavy - 1);

// voxel index along one axis: m with V[m] <= d < V[m+1], or -1 outside [V[0], V[n])
__device__ __forceinline__ int sdm_vox(float d, const float* sV, uint32_t n, float inv_w) {
  if (!(d >= sV[0]) || !(d < sV[n])) return -1;
  int m = (int)((d - sV[0]) * inv_w);
  m = m < 0 ? 0 : (m >= (int)n ? (int)n - 1 : m);
  while (m > 0 && d < sV[m]) --m;
  while (m + 1 < (int)n && d >= sV[m + 1]) ++m;
  return m;
}

// The pairs of one central (record index rec, cell ce of the neighbour grid) with the
// candidates j0 + off, j0 + off + step, ... of every stencil row.
__device__ __forceinline__ void sdm_central(const SdmArgs& a, const Geo& ng, const float* sV, float inv_w,
                                            uint32_t rec, uint32_t ce, uint32_t off, uint32_t step, uint64_t& in_map,
                                            uint64_t& outside) {
  const float4 p = __ldg(a.crec + rec);
  const uint32_t pidx = __float_as_uint(p.w);
  const int st = a.stencil;
  const uint32_t cx = ce % ng.dims[0], cy = (ce / ng.dims[0]) % ng.dims[1], cz = ce / (ng.dims[0] * ng.dims[1]);
  const uint32_t xlo = cx >= (uint32_t)st ? cx - st : 0;
  const uint32_t xhi = cx + st < ng.dims[0] ? cx + st : ng.dims[0] - 1;
  const int ylo = max((int)cy - st, 0), yhi = min((int)cy + st, (int)ng.dims[1] - 1);
  const int zlo = max((int)cz - st, 0), zhi = min((int)cz + st, (int)ng.dims[2] - 1);
  const uint32_t nv = a.n_vox;
  for (int z = zlo; z <= zhi; ++z)
    for (int y = ylo; y <= yhi; ++y) {
      const uint32_t row = ((uint32_t)z * ng.dims[1] + (uint32_t)y) * ng.dims[0];
      const uint32_t j1 = a.nstart[row + xhi + 1];
      for (uint32_t j = a.nstart[row + xlo] + off; j < j1; j += step) {
        const float4 q = __ldg(a.nrec + j);
        // the same float32 operations as the squared distance: dx = x_j - x_i
        const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 < a.ER && __float_as_uint(q.w) != pidx) {
          const int mx = sdm_vox(dx, sV, nv, inv_w), my = sdm_vox(dy, sV, nv, inv_w), mz = sdm_vox(dz, sV, nv, inv_w);
          if ((mx | my | mz) < 0) {
            ++outside;
          } else {
            atomicAdd(&a.H[((uint64_t)mz * nv + (uint64_t)my) * nv + (uint64_t)mx], 1ull);
            ++in_map;
          }
        }
      }
    }
}

__global__ void __launch_bounds__(256) k_sdm(const SdmArgs a) {
  griddep_wait();
  griddep_launch();
  __shared__ float sV[kSdmMaxVox + 1];
  __shared__ uint32_t s_rec[8][kSdmLightCap], s_cell[8][kSdmLightCap];
  for (uint32_t m = threadIdx.x; m <= a.n_vox; m += blockDim.x)
    sV[m] = __double2float_rn(__dmul_rn(__dsub_rn((double)m, (double)a.n_vox * 0.5), a.w));
  __syncthreads();
  const float inv_w = (float)(1.0 / a.w);
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Geo ng = *a.ngeo;
  uint64_t in_map = 0, outside = 0;

  // cells listed for the CTA-staged kernel (when the grid has that option): 32 centrals at a time
  const uint32_t n_dense = a.cgeo->work_n;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&a.cgeo->work_next, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_dense) break;
    const uint32_t c = a.cwork[item];
    const uint32_t c0 = a.cstart[c], n_c = a.cstart[c + 1] - c0;
    for (uint32_t b = lane; b < n_c; b += 32) sdm_central(a, ng, sV, inv_w, c0 + b, c, 0, 1, in_map, outside);
  }
  // items from the front (dense cells): the lanes take the item's centrals (one cell, so they walk
  // the same records in step); with <= 3 centrals they split each central's candidates instead
  const uint32_t n_front = a.cgeo->work_n2, n_light = a.cgeo->work_n3;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&a.cgeo->work_next2, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_front) break;
    const uint2 it = a.witem[item];
    const uint32_t c = it.x, cnt = it.y & 63u, r0 = a.cstart[c] + (it.y >> 6);
    if (cnt > 3) {
      if (lane < cnt) sdm_central(a, ng, sV, inv_w, r0 + lane, c, 0, 1, in_map, outside);
    } else {
      for (uint32_t ci = 0; ci < cnt; ++ci) sdm_central(a, ng, sV, inv_w, r0 + ci, c, lane, 32, in_map, outside);
    }
  }
  // items from the back (sparse cells), 32 at a time: their centrals are spread over the lanes
  uint32_t* rl = s_rec[w];
  uint32_t* cl = s_cell[w];
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.cgeo->work_next3, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_light) break;
    uint32_t c = 0, f = 0, cnt = 0;
    if (base + lane < n_light) {
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
    for (uint32_t q = 0; q < cnt; ++q) rl[inc - cnt + q] = f + q, cl[inc - cnt + q] = c;
    __syncwarp();
    for (uint32_t r = lane; r < total; r += 32) sdm_central(a, ng, sV, inv_w, rl[r], cl[r], 0, 1, in_map, outside);
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    in_map += __shfl_xor_sync(0xffffffffu, in_map, o);
    outside += __shfl_xor_sync(0xffffffffu, outside, o);
  }
  if (lane == 0) {
    if (in_map) atomicAdd((unsigned long long*)&a.meta[1], (unsigned long long)in_map);
    if (outside) atomicAdd((unsigned long long*)&a.meta[2], (unsigned long long)outside);
  }
}

// n_central and the device status into the meta array
__global__ void k_sdm_epilogue(const Geo* __restrict__ ngeo, const Geo* __restrict__ cgeo, uint64_t* meta) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) {
    meta[0] = cgeo->n_sel;
    int st = cgeo->status;
    if (st == 0) st = ngeo->status;
    meta[3] = (uint64_t)(uint32_t)st;
  }
}

int run_sdm(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_sdm_spec spec,
            uint64_t* d_hist, uint64_t* d_meta, cudaStream_t s) {
  const uint64_t nh = (uint64_t)spec.n_vox * spec.n_vox * spec.n_vox;
  ZeroOut z;  // the outputs are zeroed by the central-list reset kernel
  z.p[0] = d_meta;
  z.n[0] = PS_SDM_META_LEN;
  z.p[1] = d_hist;
  z.n[1] = (uint32_t)nh;
  int rc = build_central_list(g, dsrf, ctr_mask, dsrf_min, s, z);
  if (rc) return rc;
  SdmArgs a;
  memset(&a, 0, sizeof(a));
  a.nrec = g->nbr.rec;
  a.nstart = g->nbr.start;
  a.ngeo = g->nbr.geo;
  a.crec = g->ctr.rec;
  a.cstart = g->ctr.start;
  a.cwork = g->ctr.work;
  a.witem = g->ctr.witem;
  a.work_cap = g->item_cap;
  a.cgeo = g->ctr.geo;
  a.stencil = g->stencil;
  a.ER = (float)(spec.r_max * spec.r_max);
  a.w = spec.w;
  a.n_vox = spec.n_vox;
  a.H = reinterpret_cast<unsigned long long*>(d_hist);
  a.meta = d_meta;
  int per_sm = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sdm, 256, 0));
  if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "SDM kernel does not fit on an SM");
  PS_LAUNCH(PS_KID_SDM, s, PS_CUDA(launch_pdl(k_sdm, g->num_sms * per_sm, 256, 0, s, a)));
  PS_LAUNCH(PS_KID_EPILOGUE, s, PS_CUDA(launch_pdl(k_sdm_epilogue, 1, 32, 0, s, g->nbr.geo, g->ctr.geo, d_meta)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
