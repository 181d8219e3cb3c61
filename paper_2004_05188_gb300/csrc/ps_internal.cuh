// Internal definitions shared by the libps translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ps.h"

namespace ps {

constexpr uint32_t kSoftFineMax = 8192;  // fine-grid bins of the smoothed RDF
constexpr float kMinCellScale = 1.0f / 3.0f;  // cell edge / r_cut: stencils of at most 3 cells

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// device allocations of the library (live count, failure injection)
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);

void prof_begin(uint32_t kid, cudaStream_t s);
void prof_end(uint32_t kid, cudaStream_t s);
// every kernel launch of the library goes through this (launch count + optional event timing)
#define PS_LAUNCH(kid, s, ...)  \
  do {                          \
    ps::prof_begin((kid), (s)); \
    __VA_ARGS__;                \
    ps::prof_end((kid), (s));   \
  } while (0)

// Programmatic dependent launch: a kernel may be scheduled while its predecessor
// drains.  Every kernel of the library starts with griddep_wait(), which returns
// once the predecessor grid has completed and its memory is visible, so the
// order of effects is the stream order; only the launch latency overlaps.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#define PS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ps::cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// device-resident grid geometry (written by the build kernels)
// ---------------------------------------------------------------------------
struct Geo {
  float origin[3];
  float inv_h;      // 1 / cell edge, float32 (used for the cell index)
  float h;          // cell edge
  uint32_t dims[3];
  uint32_t n_cells;
  uint32_t n_sel;   // ions in the set
  int32_t bbox_key[6];  // order-preserving int keys of min xyz, max xyz
  int32_t status;   // device-side ps_status
  uint32_t work_n;     // dense cells in work[] (CTA-staged kernel)
  uint32_t work_n2;    // warp items from the front of witem[] (warp kernel)
  uint32_t work_next;  // persistent-kernel work counters
  uint32_t work_next2;
  uint32_t work_n3;    // items from the back of witem[] (sparse cells of central lists), witem[cap-1] downwards
  uint32_t work_next3; // light items taken so far (query kernel: 32 at a time)
  uint32_t work_n4;    // very heavy warp items (exact query), listed apart and taken before the others
  uint32_t work_next2b;  // second pass over the same items (the exact query's full-radius kNN fallback)
  uint32_t work_next3b;
  uint32_t sym_next;     // cells taken by the symmetric RDF pass (32 at a time)
  uint32_t list_n;       // centrals listed by the near kNN pass for the full-radius search
};

// Warp items with at least this many centrals per cell are listed first (largest work first).
constexpr uint32_t kHeavy = 16;
// Central lists: cells with fewer than kHeavy centrals and at most this many candidates in
// their stencil are "sparse" and listed from the back (one thread per central in the query).
constexpr uint32_t kSparseCand = 64;

// Lanes that share one central's candidates in the query's staged path: 1, or 2 / 4 for cells
// whose stencil holds at least 16 / 32 times the cloud's mean number of candidates (n_nbr
// records over n_cells cells, (2s+1)^3 cells per stencil), so that the items of dense
// clusters do not set the kernel's length on their own (measured on the precipitate needle:
// lower thresholds cost more instructions than the shorter tail saves, higher ones leave the
// tail).  Integer arithmetic: the central-list scan and the query compute the same value.
__host__ __device__ __forceinline__ uint32_t lanes_per_central(uint32_t n_cand, uint32_t n_nbr, uint32_t n_cells,
                                                               int stencil) {
  const uint64_t w = (uint64_t)(2 * stencil + 1) * (2 * stencil + 1) * (2 * stencil + 1);
  const uint64_t lhs = (uint64_t)n_cand * n_cells, unit = w * n_nbr;
  return lhs >= 32 * unit ? 4u : (lhs >= 16 * unit ? 2u : 1u);
}

// Lanes per central of a warp item of the exact query with cnt (4..32) centrals: the largest
// power of two, at most 8, with cnt * L <= 32.  A full item of a cell split by
// lanes_per_central (32 / L centrals) gets that L back; a cell's last, partial item gets more
// lanes, so that its warp is not left mostly idle.
__host__ __device__ __forceinline__ uint32_t item_lanes(uint32_t cnt) {
  return cnt <= 4u ? 8u : (cnt <= 8u ? 4u : (cnt <= 16u ? 2u : 1u));
}

// A warp item of the exact query is "very heavy" when each of its lanes tests at least 8 times
// the cloud's mean stencil population (n_cand / L >= 8 w n_nbr / n_cells): those items are
// listed apart and taken first, so that the query's last items are short ones (longest first).
__host__ __device__ __forceinline__ bool very_heavy(uint32_t n_cand, uint32_t L, uint32_t n_nbr, uint32_t n_cells,
                                                    int stencil) {
  const uint64_t w = (uint64_t)(2 * stencil + 1) * (2 * stencil + 1) * (2 * stencil + 1);
  return (uint64_t)n_cand * n_cells >= 8 * (uint64_t)L * w * n_nbr;
}

// item i of a list whose heavy items grow from the front and light items from the back
__device__ __forceinline__ uint2 work_item(const uint2* witem, uint32_t cap, uint32_t n_front, uint32_t i) {
  return i < n_front ? witem[i] : witem[cap - 1 - (i - n_front)];
}

// A sorted cell list: count / start per cell and the sorted records.
struct CellList {
  uint32_t* count = nullptr;   // [cell_cap]
  uint32_t* start = nullptr;   // [cell_cap + 1]
  float4* rec = nullptr;       // [n_max]: x, y, z, original index bits
  uint32_t* work = nullptr;    // [cell_cap]: dense cells
  uint2* witem = nullptr;      // [item_cap]: (cell, first central << 6 | count) warp items
  Geo* geo = nullptr;          // device
};

}  // namespace ps

struct ps_grid {
  int64_t n_max = 0;
  uint32_t cell_cap = 0;
  float cell_scale = 1.0f;
  uint32_t block = 0;
  int device = 0;
  int num_sms = 0;
  // last build
  const float* xyz = nullptr;
  const uint8_t* type = nullptr;
  int64_t n = 0;
  float r_cut = 0.0f;
  bool built = false;
  // scratch shared by both builds
  uint32_t dense_min = 0xFFFFFFFFu;  // cells with at least this many centrals go to the CTA-staged kernel
  uint32_t item_cap = 0;       // capacity of the warp item list
  int stencil = 1;             // neighbour cells searched on each side (1: cell >= r_cut, 2: cell >= r_cut/2)
  bool pack_type = false;      // records carry (index << 8 | type) instead of the index (batched sweeps)
  bool split = false;          // exact query in passes: near-radius kNN + fallback, symmetric RDF (ps_grid_opts.split)
  uint64_t nbr_mask[4] = {0, 0, 0, 0};  // type set of the last build's neighbour records
  uint32_t* sel = nullptr;     // [n_max] selected ion indices
  uint2* cr = nullptr;         // [n_max] (cell, rank) of selected ions
  unsigned long long* scan_state = nullptr;  // [scan tiles] look-back words of the single-pass scans (cells, records)
  uint32_t* scan_ctr = nullptr;              // [2] tile counter, finished-block counter
  uint32_t scan_tiles_cap = 0;
  // smoothed RDF scratch (fine grid of at most kSoftFineMax bins)
  unsigned long long* soft_m0 = nullptr;
  double* soft_m1 = nullptr;
  double* soft_m2 = nullptr;
  float* soft_T = nullptr;
  double* soft_gs = nullptr;
  uint2* nbr_witem = nullptr;  // [item_cap] warp items over the neighbour list (adjoint pass B)
  ps::CellList nbr;  // neighbour grid (geometry owner)
  ps::CellList ctr;  // central list, same geometry
  void* dev_block = nullptr;  // single allocation holding everything
};

namespace ps {

// float <-> order-preserving int key
__host__ __device__ inline int32_t f2key(float f) {
  int32_t i = 0;
#ifdef __CUDA_ARCH__
  i = __float_as_int(f);
#else
  memcpy(&i, &f, 4);
#endif
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__host__ __device__ inline float key2f(int32_t k) {
  int32_t i = k >= 0 ? k : (k ^ 0x7FFFFFFF);
  float f;
#ifdef __CUDA_ARCH__
  f = __int_as_float(i);
#else
  memcpy(&f, &i, 4);
#endif
  return f;
}

// host-side builders shared between translation units
int check_spatstat_args(const char* who, const uint64_t* ctr_mask, float dsrf_min, ps_bins bins, const uint32_t* ks,
                        uint32_t n_k, const uint64_t* d_knn, const uint64_t* d_meta, float r_cut);
int build_neighbour_grid(ps_grid* g, const uint64_t nbr_mask[4], float r_cut, cudaStream_t s);
// output arrays a central-list reset also zeroes (null pointers are skipped)
struct ZeroOut {
  uint64_t* p[3] = {nullptr, nullptr, nullptr};
  uint32_t n[3] = {0, 0, 0};
};
// split: size the warp items of dense cells for lanes_per_central (the exact query's staged path);
// vertex: centrals among the neighbour records sorted by the vertex-centred grid (the query in
// passes on cells smaller than r_cut), the central prefix in g->cr
int build_central_list(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, cudaStream_t s,
                       ZeroOut z = ZeroOut(), bool split = false, bool vertex = false);
int soft_forward(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma, float scale,
                 ps_bins bins, float* d_h, cudaStream_t s);
int run_sdm(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_sdm_spec spec,
            uint64_t* d_hist, uint64_t* d_meta, cudaStream_t s);
int run_cluster(ps_grid* g, const float* dsrf, ps_cluster_spec spec, uint32_t* d_label, uint64_t* d_size_hist,
                uint64_t* d_interior_hist, uint64_t* d_meta, cudaStream_t s);
int rdf_normalise(ps_grid* gr, const uint64_t* d_meta, const uint64_t* d_rdf, double volume, ps_bins bins,
                  double* d_g, double* d_factor, cudaStream_t s);
int soft_backward(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, float sigma, float scale,
                  ps_bins bins, const float* d_G, float* d_grad, float* d_grad_s, cudaStream_t s);

struct Mask {
  uint64_t w[4];
};

__device__ __forceinline__ bool in_mask(const Mask& m, uint32_t t) { return (m.w[t >> 6] >> (t & 63)) & 1ull; }

// cell coordinate along one axis: floor((x - origin) * inv_h), clamped to [0, dim)
__device__ __forceinline__ uint32_t cell_axis(float x, float origin, float inv_h, uint32_t dim) {
  const float u = __fmul_rn(__fsub_rn(x, origin), inv_h);
  int c = __float2int_rd(u);  // saturating; NaN -> 0
  c = c < 0 ? 0 : c;
  return (uint32_t)c >= dim ? dim - 1 : (uint32_t)c;
}

__device__ __forceinline__ uint32_t cell_of(const Geo& g, float x, float y, float z) {
  const uint32_t cx = cell_axis(x, g.origin[0], g.inv_h, g.dims[0]);
  const uint32_t cy = cell_axis(y, g.origin[1], g.inv_h, g.dims[1]);
  const uint32_t cz = cell_axis(z, g.origin[2], g.inv_h, g.dims[2]);
  return (cz * g.dims[1] + cy) * g.dims[0] + cx;
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}

// exact squared distance: float32, fixed order, no contraction
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = __fsub_rn(bx, ax);
  const float dy = __fsub_rn(by, ay);
  const float dz = __fsub_rn(bz, az);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// packed pairs of float32 (two IEEE round-to-nearest results per instruction)
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// two squared distances at once, same operation order and rounding as dist2():
// packed differences and squares, then scalar round-to-nearest additions (a packed
// add after a packed multiply can be fused into an FMA by the assembler)
__device__ __forceinline__ void dist2_x2(unsigned long long px, unsigned long long py, unsigned long long pz,
                                         unsigned long long qx, unsigned long long qy, unsigned long long qz,
                                         float& d2a, float& d2b) {
  const unsigned long long dx = f2_sub(qx, px), dy = f2_sub(qy, py), dz = f2_sub(qz, pz);
  float xa, xb, ya, yb, za, zb;
  f2_unpack(f2_mul(dx, dx), xa, xb);
  f2_unpack(f2_mul(dy, dy), ya, yb);
  f2_unpack(f2_mul(dz, dz), za, zb);
  d2a = __fadd_rn(__fadd_rn(xa, ya), za);
  d2b = __fadd_rn(__fadd_rn(xb, yb), zb);
}

// Run table of a warp: run(r, src, len) for r < n_runs (up to 64, in rounds of 32 lanes), the
// sources rsrc[r] and the prefix rpre[r + 1] of the lengths (rpre[0] = 0), so that the runs read
// as one concatenated candidate list.  Returns the total length (every lane).
template <class R>
__device__ __forceinline__ uint32_t run_table(uint32_t lane, int n_runs, uint32_t* rsrc, uint32_t* rpre, R&& run) {
  __syncwarp();
  uint32_t total = 0;
  for (int h = 0; h < n_runs; h += 32) {
    const uint32_t r = (uint32_t)h + lane;
    uint32_t src = 0, len = 0;
    if (r < (uint32_t)n_runs) run(r, src, len);
    uint32_t pre = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= (uint32_t)o) pre += y;
    }
    if (r < (uint32_t)n_runs) {
      rsrc[r] = src;
      rpre[r + 1] = total + pre;
    }
    total += __shfl_sync(0xffffffffu, pre, 31);
  }
  if (lane == 0) rpre[0] = 0;
  __syncwarp();
  return total;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk async copy (global -> shared), bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar`, giving up after `limit_ns`.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

}  // namespace ps
