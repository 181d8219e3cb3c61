// Maximum-separation clustering (Methods, "Descriptive, two-point spatial
// statistics, and clustering": the DBScan variant with the threshold distance
// d_max and the minimum cluster size N_min; the paper sweeps d_max in batch
// queues and keeps, per cluster, whether the dataset edge truncates it).
//
// Ions of the grid's set are linked when d2 <= (float)(d_max^2); the clusters
// are the connected components with at least N_min ions.  GPU form: a
// lock-free union-find over the grid's sorted records.  Every record tests the
// later records of its stencil; a link hooks the larger root under the smaller
// one with a compare-and-swap (a failed swap means another thread hooked that
// root, so every retry follows someone's progress), so each component ends
// rooted at its smallest record.  Then the paths are compressed and every
// root gathers its size, the smallest original index of its ions (the
// cluster's label) and the smallest d_srf of its ions (interior test).
// Scratch: the grid's central-list records (unused between queries).
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

struct ClusterArgs {
  const float4* rec;
  const uint32_t* start;
  const Geo* geo;
  int stencil;
  bool packed;  // record words carry (index << 8 | type)
  float D;      // (float)(d_max^2)
  uint32_t n_min;
  float dsrf_min;
  uint32_t hist_len;
  const float* dsrf;
  int64_t n;
  uint32_t* parent;
  uint32_t* size;
  uint32_t* cmin;
  int32_t* dkey;
  uint32_t* label;
  unsigned long long* size_hist;
  unsigned long long* interior_hist;
  unsigned long long* meta;
};

__device__ __forceinline__ uint32_t ld_rlx(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// root of x; shortens the path on the way (parents only ever point to smaller records, so
// replacing a parent by a grandparent keeps x in its tree)
__device__ __forceinline__ uint32_t cl_find(uint32_t* parent, uint32_t x) {
  uint32_t p = ld_rlx(parent + x);
  while (p != x) {
    const uint32_t gp = ld_rlx(parent + p);
    if (gp < p) st_rlx(parent + x, gp);
    x = p;
    p = gp;
  }
  return x;
}

__device__ __forceinline__ void cl_unite(uint32_t* parent, uint32_t a, uint32_t b) {
  a = cl_find(parent, a);
  b = cl_find(parent, b);
  while (a != b) {
    if (a > b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(parent + b, b, a);
    if (old == b) return;
    b = cl_find(parent, old);
    a = cl_find(parent, a);
  }
}

__device__ __forceinline__ uint32_t rec_index(const ClusterArgs& a, float w) {
  const uint32_t u = __float_as_uint(w);
  return a.packed ? (u >> 8) : u;
}

__global__ void __launch_bounds__(256) k_cl_init(const ClusterArgs a) {
  griddep_wait();
  griddep_launch();
  const uint32_t ns = a.geo->n_sel;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = tid; s < ns; s += stride) {
    a.parent[s] = (uint32_t)s;
    a.size[s] = 0;
    a.cmin[s] = 0xFFFFFFFFu;
    a.dkey[s] = f2key(INFINITY);
  }
  for (uint64_t i = tid; i < (uint64_t)a.n; i += stride) a.label[i] = 0xFFFFFFFFu;
  for (uint64_t b = tid; b < a.hist_len; b += stride) a.size_hist[b] = 0ull, a.interior_hist[b] = 0ull;
  if (tid < PS_CLUSTER_META_LEN) a.meta[tid] = 0ull;
}

// every record links to the later records of its stencil within d_max
__global__ void __launch_bounds__(256) k_cl_link(const ClusterArgs a) {
  griddep_wait();
  griddep_launch();
  const Geo g = *a.geo;
  const int st = a.stencil;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < g.n_sel; s += gridDim.x * blockDim.x) {
    const float4 p = __ldg(a.rec + s);
    const uint32_t c = cell_of(g, p.x, p.y, p.z);
    const uint32_t cx = c % g.dims[0], cy = (c / g.dims[0]) % g.dims[1], cz = c / (g.dims[0] * g.dims[1]);
    const uint32_t xlo = cx >= (uint32_t)st ? cx - st : 0;
    const uint32_t xhi = cx + st < g.dims[0] ? cx + st : g.dims[0] - 1;
    const int ylo = max((int)cy - st, 0), yhi = min((int)cy + st, (int)g.dims[1] - 1);
    const int zlo = max((int)cz - st, 0), zhi = min((int)cz + st, (int)g.dims[2] - 1);
    for (int z = zlo; z <= zhi; ++z)
      for (int y = ylo; y <= yhi; ++y) {
        const uint32_t row = ((uint32_t)z * g.dims[1] + (uint32_t)y) * g.dims[0];
        const uint32_t j1 = a.start[row + xhi + 1];
        uint32_t j = a.start[row + xlo];
        j = j > s ? j : s + 1;
        for (; j < j1; ++j) {
          const float4 q = __ldg(a.rec + j);
          if (dist2(p.x, p.y, p.z, q.x, q.y, q.z) <= a.D) cl_unite(a.parent, s, j);
        }
      }
  }
}

// full path compression and the per-root size, label and smallest d_srf
__global__ void __launch_bounds__(256) k_cl_gather(const ClusterArgs a) {
  griddep_wait();
  griddep_launch();
  const uint32_t ns = a.geo->n_sel;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    uint32_t r = s;
    while (a.parent[r] != r) r = a.parent[r];
    a.parent[s] = r;
    const uint32_t idx = rec_index(a, __ldg(a.rec + s).w);
    atomicAdd(a.size + r, 1u);
    atomicMin(a.cmin + r, idx);
    if (a.dsrf) atomicMin(a.dkey + r, f2key(a.dsrf[idx]));
  }
}

// labels in original index order, histograms of the cluster sizes, counters
__global__ void __launch_bounds__(256) k_cl_final(const ClusterArgs a) {
  griddep_wait();
  griddep_launch();
  const uint32_t ns = a.geo->n_sel;
  unsigned long long n_cl = 0, n_in = 0, n_int = 0;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const uint32_t r = a.parent[s];
    const uint32_t sz = a.size[r];
    if (sz < a.n_min) continue;
    a.label[rec_index(a, __ldg(a.rec + s).w)] = a.cmin[r];
    if (r != s) continue;
    const uint32_t b = sz >= a.hist_len - 1 ? a.hist_len - 1 : sz;
    atomicAdd(a.size_hist + b, 1ull);
    ++n_cl;
    n_in += sz;
    if (key2f(a.dkey[r]) >= a.dsrf_min) {
      atomicAdd(a.interior_hist + b, 1ull);
      ++n_int;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_cl += __shfl_xor_sync(0xffffffffu, n_cl, o);
    n_in += __shfl_xor_sync(0xffffffffu, n_in, o);
    n_int += __shfl_xor_sync(0xffffffffu, n_int, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_cl) atomicAdd(a.meta + 1, n_cl);
    if (n_in) atomicAdd(a.meta + 2, n_in);
    if (n_int) atomicAdd(a.meta + 3, n_int);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.meta[0] = ns;
    a.meta[4] = (unsigned long long)(uint32_t)a.geo->status;
  }
}

int run_cluster(ps_grid* g, const float* dsrf, ps_cluster_spec spec, uint32_t* d_label, uint64_t* d_size_hist,
                uint64_t* d_interior_hist, uint64_t* d_meta, cudaStream_t s) {
  ClusterArgs a;
  memset(&a, 0, sizeof(a));
  a.rec = g->nbr.rec;
  a.start = g->nbr.start;
  a.geo = g->nbr.geo;
  a.stencil = g->stencil;
  a.packed = g->pack_type;
  a.D = (float)(spec.d_max * spec.d_max);
  a.n_min = spec.n_min;
  a.dsrf_min = spec.dsrf_min;
  a.hist_len = spec.hist_len;
  a.dsrf = dsrf;
  a.n = g->n;
  // scratch: the central-list records, 16 B per ion of capacity
  uint32_t* scratch = reinterpret_cast<uint32_t*>(g->ctr.rec);
  const size_t nm = (size_t)g->n_max;
  a.parent = scratch;
  a.size = scratch + nm;
  a.cmin = scratch + 2 * nm;
  a.dkey = reinterpret_cast<int32_t*>(scratch + 3 * nm);
  a.label = d_label;
  a.size_hist = reinterpret_cast<unsigned long long*>(d_size_hist);
  a.interior_hist = reinterpret_cast<unsigned long long*>(d_interior_hist);
  a.meta = reinterpret_cast<unsigned long long*>(d_meta);
  const int blocks = g->num_sms * 8;
  PS_LAUNCH(PS_KID_CLUSTER, s, PS_CUDA(launch_pdl(k_cl_init, blocks, 256, 0, s, a)));
  PS_LAUNCH(PS_KID_CLUSTER, s, PS_CUDA(launch_pdl(k_cl_link, blocks, 256, 0, s, a)));
  PS_LAUNCH(PS_KID_CLUSTER, s, PS_CUDA(launch_pdl(k_cl_gather, blocks, 256, 0, s, a)));
  PS_LAUNCH(PS_KID_CLUSTER, s, PS_CUDA(launch_pdl(k_cl_final, blocks, 256, 0, s, a)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
