// Randomised type labels: the companion statistic the paper computes by
// default next to every spatial statistic, with the type labels shuffled by a
// pseudo-random generator (Suppl. "Importance of high quality random number
// generators") so that the result can be compared with a random arrangement.
//
// GPU form: no sort.  perm is a pseudo-random permutation of [0, n) that every
// thread evaluates on its own: a 4-round Feistel network on 2h bits
// (2^(2h) >= n) whose round function is the splitmix64 finaliser of
// (half-block + round key), round key r = finaliser(seed + (r + 1) * golden
// gamma), restricted to [0, n) by cycle walking.  type_out[i] = type_in[perm(i)].
#include "ps_internal.cuh"

namespace ps {

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

struct FeistelKey {
  uint64_t k[4];
  uint32_t h;
};

__device__ __forceinline__ uint64_t feistel4(uint64_t x, const FeistelKey& key) {
  const uint64_t mask = (1ull << key.h) - 1ull;
  uint64_t L = x >> key.h, R = x & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t t = L ^ (sm_mix(R + key.k[r]) & mask);
    L = R;
    R = t;
  }
  return (L << key.h) | R;
}

__global__ void __launch_bounds__(256) k_shuffle_labels(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                        uint32_t* __restrict__ perm, uint64_t n, FeistelKey key,
                                                        int* __restrict__ status) {
  griddep_wait();
  griddep_launch();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t domain = 1ull << (2 * key.h);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t y = feistel4(i, key);
    // cycle walking: the cycle through i returns below n within `domain` steps
    for (uint64_t w = 0; y >= n && w < domain; ++w) y = feistel4(y, key);
    if (y >= n) {  // not reachable for a permutation; never read out of bounds
      if (status) atomicCAS(status, 0, (int)PS_ERR_INVALID_INPUT);
      y = i;
    }
    out[i] = in[y];
    if (perm) perm[i] = (uint32_t)y;
  }
}

}  // namespace ps

using namespace ps;

extern "C" int ps_shuffle_labels(const uint8_t* type_in, uint8_t* type_out, int64_t n, uint64_t seed, uint32_t* d_perm,
                                 void* stream) {
  if (n < 0 || n > (int64_t)UINT32_MAX) return fail(PS_ERR_INVALID_ARG, "ps_shuffle_labels: n out of range");
  if (n > 0 && (!type_in || !type_out)) return fail(PS_ERR_INVALID_ARG, "ps_shuffle_labels: NULL array");
  if (n > 0 && type_in == type_out) return fail(PS_ERR_INVALID_ARG, "ps_shuffle_labels: in and out must differ");
  if (n == 0) return PS_OK;
  FeistelKey key;
  key.h = 1;
  while ((1ull << (2 * key.h)) < (uint64_t)n) ++key.h;
  for (int r = 0; r < 4; ++r) key.k[r] = sm_mix(seed + (uint64_t)(r + 1) * 0x9e3779b97f4a7c15ULL);
  int dev = 0, sms = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PS_LAUNCH(PS_KID_LABELS, s,
            PS_CUDA(launch_pdl(k_shuffle_labels, sms * 8, 256, 0, s, type_in, type_out, d_perm, (uint64_t)n, key,
                               static_cast<int*>(nullptr))));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}
