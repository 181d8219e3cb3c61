// Throughput microbenchmarks of the units the statistics are bound by: the
// denominators of their rooflines, measured on the GPU at hand instead of
// taken from data sheets.
//   FP32 add / multiply (not fused), scalar and packed f32x2: the pair test
//     of the query is ((dx*dx)+(dy*dy))+(dz*dz) with no contraction;
//   32-bit shared-memory atomic adds to distinct banks: the RDF histograms;
//   the SM clock during the runs (clock64 ticks per %globaltimer ns).
// Independent dependency chains, no multiply feeding an add (nothing the
// compiler could contract), results kept live through a store that never runs.
#include "ps_internal.cuh"

namespace ps {

constexpr int kPeakThreads = 1024;

__device__ __forceinline__ void clock_probe(unsigned long long* clk) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64();
    clk[1] = global_ns();
  }
}
__device__ __forceinline__ void clock_probe_end(unsigned long long* clk) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[2] = clock64();
    clk[3] = global_ns();
  }
}

// 8 multiply chains and 8 add chains per thread, 16 float32 results per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_fp32_scalar(float* sink, int iters, float c, float d,
                                                                   unsigned long long* clk) {
  clock_probe(clk);
  float m[8], a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) m[k] = 1.0f + 1e-3f * (threadIdx.x + k), a[k] = (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      m[k] = __fmul_rn(m[k], c);
      a[k] = __fadd_rn(a[k], d);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += m[k] + a[k];
  if (s == -1.0f) sink[threadIdx.x] = s;
  clock_probe_end(clk);
}

// the same with packed pairs: 4 multiply and 4 add f32x2 chains, 16 results per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_fp32_packed(float* sink, int iters, float c, float d,
                                                                   unsigned long long* clk) {
  clock_probe(clk);
  unsigned long long m[4], a[4];
  const unsigned long long cc = f2_pack(c, c), dd = f2_pack(d, d);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    m[k] = f2_pack(1.0f + 1e-3f * (threadIdx.x + k), 1.0f - 1e-3f * k), a[k] = f2_pack((float)k, 0.5f * k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m[k] = f2_mul(m[k], cc);
      a[k] = f2_add(a[k], dd);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float x, y, u, v;
    f2_unpack(m[k], x, y);
    f2_unpack(a[k], u, v);
    s += x + y + u + v;
  }
  if (s == -1.0f) sink[threadIdx.x] = s;
  clock_probe_end(clk);
}

// shared-memory atomic adds without return, every thread on its own word (distinct banks in a warp)
__global__ void __launch_bounds__(kPeakThreads) k_peak_smem_atomic(uint32_t* sink, int iters,
                                                                   unsigned long long* clk) {
  clock_probe(clk);
  __shared__ uint32_t s[kPeakThreads];
  s[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t addr = smem_u32(&s[threadIdx.x]);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
  }
  __syncthreads();
  if (s[threadIdx.x] == 0xFFFFFFFFu) sink[threadIdx.x] = s[threadIdx.x];
  clock_probe_end(clk);
}

}  // namespace ps

using namespace ps;

extern "C" int ps_measure_peaks(ps_peaks* out, void* stream) {
  if (!out || out->struct_size < sizeof(ps_peaks)) return fail(PS_ERR_INVALID_ARG, "ps_measure_peaks: out/struct_size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // scratch for the sinks and the clock probe (freed before returning)
  void* buf = nullptr;
  PS_CUDA(dev_malloc(&buf, kPeakThreads * 4 + 64));
  float* sink = static_cast<float*>(buf);
  unsigned long long* clk = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + kPeakThreads * 4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PS_OK;
  double best[3] = {0, 0, 0}, mhz = 0.0;
  const int blocks = sms * 2;
  const int it_fp = 1 << 15, it_at = 1 << 12;
  const double threads = (double)blocks * kPeakThreads;
  const double work[3] = {threads * it_fp * 16.0, threads * it_fp * 16.0, threads * it_at * 8.0};
  auto done = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == PS_OK) rc = cuda_fail(e, what);
    return rc == PS_OK;
  };
  if (done(cudaEventCreate(&e0), "cudaEventCreate") && done(cudaEventCreate(&e1), "cudaEventCreate")) {
    for (int rep = 0; rep < 3 && rc == PS_OK; ++rep) {
      for (int k = 0; k < 3 && rc == PS_OK; ++k) {
        done(cudaEventRecord(e0, s), "cudaEventRecord");
        PS_LAUNCH(PS_KID_PEAKS, s, {
          if (k == 0) k_peak_fp32_scalar<<<blocks, kPeakThreads, 0, s>>>(sink, it_fp, 0.99999994f, 1e-7f, clk);
          if (k == 1) k_peak_fp32_packed<<<blocks, kPeakThreads, 0, s>>>(sink, it_fp, 0.99999994f, 1e-7f, clk);
          if (k == 2) k_peak_smem_atomic<<<blocks, kPeakThreads, 0, s>>>(reinterpret_cast<uint32_t*>(sink), it_at, clk);
        });
        done(cudaGetLastError(), "peak kernel launch");
        done(cudaEventRecord(e1, s), "cudaEventRecord");
        done(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        if (rc == PS_OK && done(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime") && ms > 0.f)
          best[k] = fmax(best[k], work[k] / (ms * 1e-3));
        unsigned long long h[4] = {0, 0, 0, 0};
        if (rc == PS_OK && done(cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost), "cudaMemcpy") && h[3] > h[1])
          mhz = fmax(mhz, (double)(h[2] - h[0]) / (double)(h[3] - h[1]) * 1e3);
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(buf);
  if (rc) return rc;
  out->num_sms = sms;
  out->fp32_scalar_gops = best[0] * 1e-9;
  out->fp32_packed_gops = best[1] * 1e-9;
  out->smem_atomic_gops = best[2] * 1e-9;
  out->sm_mhz = mhz;
  return PS_OK;
}
