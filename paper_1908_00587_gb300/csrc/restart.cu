// Restart with a change of resolution (Sec. 2.1: at a restart the spatial
// resolution may change, by interpolation and mode padding).
//
// A state of another run of the same gap and axial period is mapped onto this
// context's grid:
//   * radial: the polynomial of degree Nr_src - 1 through the source's nodal
//     values (Chebyshev-Gauss-Lobatto nodes, wall nodes included) evaluated
//     at this grid's nodes.  The interpolation matrix is built on the host in
//     the barycentric form for those nodes, weights (-1)^j (1/2 at the ends):
//     the nodes are an affine image of the Chebyshev extreme points, which
//     leaves the weights unchanged up to a common factor.  Coinciding nodes
//     (the walls) give rows of the identity, so wall values copy exactly;
//   * Fourier: modes held by both runs are copied, modes only this run holds
//     are zero, modes only the source holds are dropped;
//   * temperature: a source without T gets this run's conductive profile; a
//     source with T given to a run without it loses T.
// One thread per destination coefficient; each sums over the source's
// radial nodes.  This runs once per restart, not per step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "tc_internal.h"

namespace tc {
namespace {

__global__ void k_regrid(const double2 *__restrict__ src, double2 *__restrict__ dst,
                         const double *__restrict__ P, Sizes s, int nf_copy, int Nr_src,
                         int M_src, int K_src) {
  const long long n = (long long)nf_copy * s.S;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int f = (int)(i / s.S);
  const long long rem = i - (long long)f * s.S;
  const int j = (int)(rem / s.nmode);
  const int mode = (int)(rem - (long long)j * s.nmode);
  const int m = mode / s.NK, kk = mode % s.NK;
  const int kv = kk <= s.K ? kk : kk - s.NK;
  double2 acc = {0.0, 0.0};
  if (m <= M_src && kv <= K_src && -kv <= K_src) {
    const int NK_src = 2 * K_src + 1;
    const long long nmode_src = (long long)(M_src + 1) * NK_src;
    const int kk_src = kv >= 0 ? kv : NK_src + kv;
    const double2 *col = src + (long long)f * Nr_src * nmode_src + (long long)m * NK_src + kk_src;
    const double *row = P + (long long)j * Nr_src;
    for (int q = 0; q < Nr_src; ++q) {
      const double w = row[q];
      const double2 x = col[q * nmode_src];
      acc.x += w * x.x;
      acc.y += w * x.y;
    }
  }
  dst[i] = acc;
}

// Barycentric interpolation matrix from the source's CGL radii to this grid's.
std::vector<double> interp_matrix(const tc_ctx *c, int Nr_src) {
  std::vector<double> rs(Nr_src), wt(Nr_src);
  for (int q = 0; q < Nr_src; ++q) {
    rs[q] = c->r_i + 0.5 * (1.0 - std::cos(M_PI * (double)q / (double)(Nr_src - 1)));
    wt[q] = ((q % 2) ? -1.0 : 1.0) * ((q == 0 || q == Nr_src - 1) ? 0.5 : 1.0);
  }
  const int Nr = c->sz.Nr;
  std::vector<double> P((size_t)Nr * Nr_src, 0.0);
  for (int j = 0; j < Nr; ++j) {
    const double x = c->r[j];
    int hit = -1;
    for (int q = 0; q < Nr_src; ++q)
      if (x == rs[q]) hit = q;
    double *row = &P[(size_t)j * Nr_src];
    if (hit >= 0) {
      row[hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int q = 0; q < Nr_src; ++q) {
      row[q] = wt[q] / (x - rs[q]);
      den += row[q];
    }
    for (int q = 0; q < Nr_src; ++q) row[q] /= den;
  }
  return P;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_set_state_regrid(tc_ctx *c, const void *spec, int Nr_src, int M_src,
                                         int K_src, int nfields_src, double eta_src,
                                         double Lz_src, int where) {
  if (!c || !spec || (where != 0 && where != 1)) return TC_ERR_ARG;
  if (Nr_src < 2 || Nr_src > 4096 || M_src < 0 || K_src < 0 || M_src > 4096 || K_src > 4096 ||
      (nfields_src != 3 && nfields_src != 4))
    return TC_ERR_ARG;
  if (!(std::fabs(eta_src - c->eta) <= 1e-14 * c->eta) ||
      !(std::fabs(Lz_src - c->Lz) <= 1e-14 * c->Lz))
    return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const Sizes &s = c->sz;
  const size_t src_bytes =
      (size_t)16 * nfields_src * Nr_src * (size_t)(M_src + 1) * (size_t)(2 * K_src + 1);
  const std::vector<double> P = interp_matrix(c, Nr_src);
  double2 *src_dev = nullptr;
  double *P_dev = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(c->stream);
    if (where == 0 && src_dev) cudaFree(src_dev);
    if (P_dev) cudaFree(P_dev);
  };
  if (over_budget(c, (where == 0 ? src_bytes : 0) + P.size() * sizeof(double)))
    return TC_ERR_OOM;
  cudaError_t e = cudaSuccess;
  if (where == 0) {
    e = cudaMalloc(&src_dev, src_bytes);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(src_dev, spec, src_bytes, cudaMemcpyHostToDevice, c->stream);
  } else {
    src_dev = const_cast<double2 *>(static_cast<const double2 *>(spec));
  }
  if (e == cudaSuccess) e = cudaMalloc(&P_dev, P.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P_dev, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream);
  if (e != cudaSuccess) {
    release();
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA;
  }
  const int nf_copy = nfields_src < s.nf ? nfields_src : s.nf;
  const long long n = (long long)nf_copy * s.S;
  {
    LaunchScope ls(c, KREGRID);
    k_regrid<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(src_dev, c->Xp, P_dev, s, nf_copy,
                                                                 Nr_src, M_src, K_src);
  }
  if (s.nf == 4 && nfields_src == 3)   // conductive temperature of this run
    e = cudaMemcpyAsync(c->Xp + 3 * s.S, c->base_dev + 3 * s.S, (size_t)16 * s.S,
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  release();
  if (e != cudaSuccess) {
    c->poisoned = true;
    std::fprintf(stderr, "libtc: regrid: %s\n", cudaGetErrorString(e));
    return TC_ERR_CUDA;
  }
  return commit_staged_state(c);
}
