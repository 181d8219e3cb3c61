// Allocation-free exact kNN + RDF: the grid scratch lives in a file-scope
// device array instead of memory from cudaMalloc.
//
// Who needs this: callers that cannot allocate device memory when they run the
// statistics, for example applications that hand all device memory to their
// own pool at start-up (so a cudaMalloc inside the library would fail), and
// long-running acquisition or visualisation loops that must not block on the
// device-wide synchronisation that cudaMalloc/cudaFree imply.
//
// The array is sized for PS_STATIC_MAX_IONS ions (about 14 MB) and every
// process that loads libps holds it on each GPU it uses until exit.
#include <cmath>
#include <mutex>

#include "ps_internal.cuh"

namespace ps {

int run_query(ps_grid* g, const float* dsrf, const uint64_t ctr_mask[4], float dsrf_min, ps_bins bins,
              const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn, uint64_t* d_meta, float* d_kth,
              uint32_t* d_nwithin, cudaStream_t s);

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kN = PS_STATIC_MAX_IONS;
constexpr size_t kCells = kN / 8 > 65536 ? kN / 8 : 65536;  // same cell capacity rule as ps_grid_create
constexpr size_t kTiles = ((kCells > kN + 1 ? kCells : kN + 1) + 4095) / 4096;  // cells or records
constexpr size_t kItems = kCells + kN / 8 + 2;  // same item capacity rule as ps_grid_create

// byte offsets of every scratch buffer inside the array
constexpr size_t o_sel = 0;
constexpr size_t o_cr = o_sel + align256(kN * 4);
constexpr size_t o_ncount = o_cr + align256(kN * 8);
constexpr size_t o_nstart = o_ncount + align256(kCells * 4);
constexpr size_t o_nrec = o_nstart + align256((kCells + 1) * 4);
constexpr size_t o_ccount = o_nrec + align256(kN * 16);
constexpr size_t o_cstart = o_ccount + align256(kCells * 4);
constexpr size_t o_crec = o_cstart + align256((kCells + 1) * 4);
constexpr size_t o_cwork = o_crec + align256(kN * 16);
constexpr size_t o_witem = o_cwork + align256(kCells * 4);
constexpr size_t o_nwitem = o_witem + align256(kItems * 8);  // very heavy items of the query
constexpr size_t o_part = o_nwitem + align256(kItems * 8);
constexpr size_t o_sctr = o_part + align256(kTiles * 8);
constexpr size_t o_ngeo = o_sctr + align256(8);
constexpr size_t o_cgeo = o_ngeo + align256(sizeof(Geo));
constexpr size_t kBytes = o_cgeo + align256(sizeof(Geo));

constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

}  // namespace

// The scratch.  In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kBytes];

}  // namespace ps

using namespace ps;

extern "C" int ps_spatstat_static(const float* xyz, const uint8_t* type, const float* dsrf, int64_t n,
                                  const uint64_t nbr_mask[4], float r_cut, const uint64_t ctr_mask[4], float dsrf_min,
                                  ps_bins bins, const uint32_t* ks, uint32_t n_k, uint64_t* d_rdf, uint64_t* d_knn,
                                  uint64_t* d_meta, float* d_kth, uint32_t* d_nwithin, void* stream) {
  if (n < 0) return fail(PS_ERR_INVALID_ARG, "ps_spatstat_static: n < 0");
  if (n > (int64_t)PS_STATIC_MAX_IONS)
    return fail(PS_ERR_CAPACITY, "ps_spatstat_static: n exceeds PS_STATIC_MAX_IONS (262144); use ps_build_grid");
  // every argument check of the build and of the statistics comes first: a refused call
  // enqueues nothing and leaves the shared scratch as it was
  if (n > 0 && (!xyz || !type)) return fail(PS_ERR_INVALID_ARG, "ps_spatstat_static: xyz/type is NULL");
  if (!nbr_mask) return fail(PS_ERR_INVALID_ARG, "ps_spatstat_static: nbr_mask is NULL");
  if (!(r_cut > 0.0f) || !std::isfinite(r_cut)) return fail(PS_ERR_INVALID_ARG, "ps_spatstat_static: r_cut must be > 0");
  int rc = check_spatstat_args("ps_spatstat_static", ctr_mask, dsrf_min, bins, ks, n_k, d_knn, d_meta, r_cut);
  if (rc) return rc;
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PS_ERR_UNSUPPORTED, "ps_spatstat_static: device index too large");
  void* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) {
      // first call on this device (the device is current): resolve the array's device address
      void* p = nullptr;
      PS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
      int m = 0;
      PS_CUDA(cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev));
      g_addr[dev] = p;
      g_sms[dev] = m;
    }
    base = g_addr[dev];
    sms = g_sms[dev];
  }
  char* b = static_cast<char*>(base);
  ps_grid g;  // a grid whose scratch is the static array (nothing to free)
  g.n_max = (int64_t)kN;
  g.cell_cap = (uint32_t)kCells;
  g.cell_scale = 1.0f;
  g.stencil = 1;
  g.item_cap = (uint32_t)kItems;
  g.scan_tiles_cap = (uint32_t)kTiles;
  g.device = dev;
  g.num_sms = sms;
  g.sel = reinterpret_cast<uint32_t*>(b + o_sel);
  g.cr = reinterpret_cast<uint2*>(b + o_cr);
  g.nbr.count = reinterpret_cast<uint32_t*>(b + o_ncount);
  g.nbr.start = reinterpret_cast<uint32_t*>(b + o_nstart);
  g.nbr.rec = reinterpret_cast<float4*>(b + o_nrec);
  g.nbr.geo = reinterpret_cast<Geo*>(b + o_ngeo);
  g.ctr.count = reinterpret_cast<uint32_t*>(b + o_ccount);
  g.ctr.start = reinterpret_cast<uint32_t*>(b + o_cstart);
  g.ctr.rec = reinterpret_cast<float4*>(b + o_crec);
  g.ctr.work = reinterpret_cast<uint32_t*>(b + o_cwork);
  g.ctr.witem = reinterpret_cast<uint2*>(b + o_witem);
  g.nbr_witem = reinterpret_cast<uint2*>(b + o_nwitem);
  g.ctr.geo = reinterpret_cast<Geo*>(b + o_cgeo);
  g.scan_state = reinterpret_cast<unsigned long long*>(b + o_part);  // zero at load; each scan clears it again
  g.scan_ctr = reinterpret_cast<uint32_t*>(b + o_sctr);
  // The build kernels clear every counter and geometry field before use, so the
  // previous call's contents never leak into this one.
  rc = ps_grid_build(&g, xyz, type, n, nbr_mask, r_cut, stream);
  if (rc) return rc;
  return ps_spatstat(&g, dsrf, ctr_mask, dsrf_min, bins, ks, n_k, d_rdf, d_knn, d_meta, d_kth, d_nwithin, stream);
}
