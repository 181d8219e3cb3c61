// Internal definitions shared by the libps translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ps.h"

namespace ps {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

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
  uint32_t work_n;  // non-empty cells in the work list
  uint32_t work_next;  // persistent-kernel work counter
  uint32_t pad[2];
};

// A sorted cell list: count / start per cell and the sorted records.
struct CellList {
  uint32_t* count = nullptr;   // [cell_cap]
  uint32_t* start = nullptr;   // [cell_cap + 1]
  float4* rec = nullptr;       // [n_max]: x, y, z, original index bits
  uint32_t* work = nullptr;    // [cell_cap]: non-empty cells
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
  uint32_t* sel = nullptr;     // [n_max] selected ion indices
  uint2* cr = nullptr;         // [n_max] (cell, rank) of selected ions
  uint32_t* scan_part = nullptr;  // [scan tiles]
  uint32_t scan_tiles_cap = 0;
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
int build_neighbour_grid(ps_grid* g, const uint64_t nbr_mask[4], float r_cut, cudaStream_t s);
int build_central_list(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, cudaStream_t s);

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
