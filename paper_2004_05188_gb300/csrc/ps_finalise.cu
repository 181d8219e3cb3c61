// Normalised RDF g(r): the finalisation of the integer RDF histogram.
//
// The paper names the RDF as the distribution of neighbours in radial shells
// about every central ion (Methods, "Descriptive, two-point spatial
// statistics, and clustering") and reports it normalised, without a formula.
// Reading: the count of bin b is divided by the count a uniform neighbour
// density rho = |N| / V puts in that shell about each of the |C| centrals,
//   g_b = H[b] / (|C| rho 4/3 pi (e_{b+1}^3 - e_b^3)),  e_b = r0 + b dr,
// in FP64 on the device, with |C| from the meta array of the query and |N|
// from the grid's neighbour set (no host synchronisation).
#include "ps_internal.cuh"

namespace ps {

__global__ void k_rdf_normalise(const Geo* __restrict__ ngeo, const uint64_t* __restrict__ meta,
                                const uint64_t* __restrict__ rdf, double r0, double dr, uint32_t n_bins,
                                double volume, double* __restrict__ g, double* __restrict__ factor) {
  griddep_wait();
  griddep_launch();
  const double nc = (double)meta[PS_META_N_CENTRAL];
  const double rho = __ddiv_rn((double)ngeo->n_sel, volume);
  const double c43pi = 4.0 / 3.0 * 3.14159265358979323846;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
    const double e0 = __dadd_rn(r0, __dmul_rn((double)b, dr));
    const double e1 = __dadd_rn(r0, __dmul_rn((double)(b + 1), dr));
    const double cube = __dsub_rn(__dmul_rn(__dmul_rn(e1, e1), e1), __dmul_rn(__dmul_rn(e0, e0), e0));
    const double expected = __dmul_rn(__dmul_rn(nc, rho), __dmul_rn(c43pi, cube));
    if (factor) factor[b] = expected > 0.0 ? __ddiv_rn(1.0, expected) : 0.0;
    if (g) g[b] = expected > 0.0 ? __ddiv_rn((double)rdf[b], expected) : 0.0;
  }
}

int rdf_normalise(ps_grid* gr, const uint64_t* d_meta, const uint64_t* d_rdf, double volume, ps_bins bins,
                  double* d_g, double* d_factor, cudaStream_t s) {
  const uint32_t blocks = (bins.n_bins + 255) / 256;
  PS_LAUNCH(PS_KID_FINALISE, s,
            PS_CUDA(launch_pdl(k_rdf_normalise, blocks, 256, 0, s, gr->nbr.geo, d_meta, d_rdf, bins.r0, bins.dr,
                               bins.n_bins, volume, d_g, d_factor)));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
