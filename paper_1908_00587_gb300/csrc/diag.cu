// Diagnostics: energy, dissipation, torque, wall power, buoyancy work,
// Nusselt number (paper Sec. 4: heat flux at the inner wall over that of the
// conductive basic state) and divergence, from the spectral state.
//
// Integrals over theta and z are Parseval sums over the stored half plane
// (weight 1 for m = 0, 2 for m > 0); the radial integral uses Clenshaw-Curtis
// weights times r.  One CTA per radial level reduces over modes in a fixed
// order; one thread then sums the levels in order, so results are
// deterministic run to run.
#include <cuda_runtime.h>

#include <algorithm>

#include "tc_internal.h"

namespace tc {

namespace {

constexpr int kDiagThreads = 256;
constexpr int kNPart = 6;   // E, E_pert, 2S:S, u_z T, |div|^2, max |div|

__device__ __forceinline__ double n2(double2 a) { return a.x * a.x + a.y * a.y; }

__global__ void k_diag_level(const double2 *__restrict__ X, const double2 *__restrict__ base,
                             double *__restrict__ part, Sizes s, Radial rad, double alpha) {
  const int j = blockIdx.x;
  const double ir = rad.inv_r[j];
  const int st = rad.s0[j];
  const double *d1 = rad.D1 + j * kStencil;
  double acc[kNPart] = {0, 0, 0, 0, 0, 0};
  for (int mode = threadIdx.x; mode < s.nmode; mode += blockDim.x) {
    const int m = mode / s.NK, kk = mode % s.NK;
    const int kv = kk <= s.K ? kk : kk - s.NK;
    const double beta = alpha * kv;
    const double cm = (m == 0) ? 1.0 : 2.0;
    const long long i = (long long)j * s.nmode + mode;
    const double2 ur = X[i], ut = X[s.S + i], uz = X[2 * s.S + i];
    double2 dr_ur = {0, 0}, dr_ut = {0, 0}, dr_uz = {0, 0}, dr_rur = {0, 0};
#pragma unroll
    for (int t = 0; t < kStencil; ++t) {
      const long long o = (long long)(st + t) * s.nmode + mode;
      const double2 a = X[o], b = X[s.S + o], c = X[2 * s.S + o];
      const double w = d1[t], rw = d1[t] * rad.r[st + t];
      dr_ur.x += w * a.x; dr_ur.y += w * a.y;
      dr_ut.x += w * b.x; dr_ut.y += w * b.y;
      dr_uz.x += w * c.x; dr_uz.y += w * c.y;
      dr_rur.x += rw * a.x; dr_rur.y += rw * a.y;
    }
    double2 d0 = ur, d1v = ut, d2 = uz;
    if (mode == 0) {
      const double2 b0 = base[i], b1 = base[s.S + i], b2 = base[2 * s.S + i];
      d0 = {ur.x - b0.x, ur.y - b0.y};
      d1v = {ut.x - b1.x, ut.y - b1.y};
      d2 = {uz.x - b2.x, uz.y - b2.y};
    }
    acc[0] += cm * (n2(ur) + n2(ut) + n2(uz));
    acc[1] += cm * (n2(d0) + n2(d1v) + n2(d2));
    const double fm = (double)m;
    const double2 Srr = dr_ur;
    const double2 Stt = {-fm * ut.y * ir + ur.x * ir, fm * ut.x * ir + ur.y * ir};
    const double2 Szz = {-beta * uz.y, beta * uz.x};
    const double2 Srt = {0.5 * (dr_ut.x - ut.x * ir - fm * ur.y * ir),
                         0.5 * (dr_ut.y - ut.y * ir + fm * ur.x * ir)};
    const double2 Srz = {0.5 * (-beta * ur.y + dr_uz.x), 0.5 * (beta * ur.x + dr_uz.y)};
    const double2 Stz = {0.5 * (-beta * ut.y - fm * uz.y * ir), 0.5 * (beta * ut.x + fm * uz.x * ir)};
    acc[2] += cm * (2.0 * (n2(Srr) + n2(Stt) + n2(Szz)) + 4.0 * (n2(Srt) + n2(Srz) + n2(Stz)));
    if (s.nf == 4) {
      const double2 T = X[3 * s.S + i];
      acc[3] += cm * (uz.x * T.x + uz.y * T.y);
    }
    const double2 dv = {dr_rur.x * ir - fm * ut.y * ir - beta * uz.y,
                        dr_rur.y * ir + fm * ut.x * ir + beta * uz.x};
    acc[4] += cm * n2(dv);
    acc[5] = fmax(acc[5], sqrt(n2(dv)));
  }
  __shared__ double sh[kNPart][kDiagThreads];
#pragma unroll
  for (int q = 0; q < kNPart; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int q = 0; q < kNPart - 1; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
      sh[kNPart - 1][threadIdx.x] = fmax(sh[kNPart - 1][threadIdx.x], sh[kNPart - 1][threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x < kNPart) part[j * kNPart + threadIdx.x] = sh[threadIdx.x][0];
}

// out: t-less tc_diag fields in order dt, E, E_pert, torque_i, torque_o, P_wall,
// eps, buoy_work, Nu_i, Nu_o, div_max, div_rms, cfl
__global__ void k_diag_final(const double2 *__restrict__ X, const double *__restrict__ part,
                             const double *__restrict__ Tb, double *__restrict__ out, Sizes s,
                             Radial rad, double V, double Gr, double Re_i, double Re_o,
                             const DevScalars *sc) {
  double E = 0, Ep = 0, ss = 0, bw = 0, dv2 = 0, dvmax = 0, vol = 0;
  for (int j = 0; j < s.Nr; ++j) {
    const double w = rad.wr[j];
    E += w * part[j * kNPart + 0];
    Ep += w * part[j * kNPart + 1];
    ss += w * part[j * kNPart + 2];
    bw += w * part[j * kNPart + 3];
    dv2 += w * part[j * kNPart + 4];
    dvmax = fmax(dvmax, part[j * kNPart + 5]);
    vol += w;
  }
  // mean-flow wall stress d u_theta/dr - u_theta/r at both walls
  double sig[2], dT[2] = {0, 0}, dTb[2] = {1, 1};
  for (int w = 0; w < 2; ++w) {
    const int j = (w == 0) ? 0 : s.Nr - 1;
    const int st = rad.s0[j];
    double du = 0, dt_ = 0, dtb = 0;
    for (int t = 0; t < kStencil; ++t) {
      const long long o = (long long)(st + t) * s.nmode;
      du += rad.D1[j * kStencil + t] * X[s.S + o].x;
      if (s.nf == 4) {
        dt_ += rad.D1[j * kStencil + t] * X[3 * s.S + o].x;
        dtb += rad.D1[j * kStencil + t] * Tb[st + t];
      }
    }
    sig[w] = du - X[s.S + (long long)j * s.nmode].x * rad.inv_r[j];
    dT[w] = dt_;
    dTb[w] = dtb;
  }
  const double ri = rad.r[0], ro = rad.r[s.Nr - 1];
  out[0] = sc->dt;
  out[1] = 0.5 * V * E;
  out[2] = 0.5 * V * Ep;
  out[3] = V * ri * ri * sig[0];
  out[4] = V * ro * ro * sig[1];
  out[5] = V * (ro * Re_o * sig[1] - ri * Re_i * sig[0]);
  out[6] = V * ss;
  out[7] = (s.nf == 4) ? Gr * V * bw : 0.0;
  out[8] = (s.nf == 4) ? dT[0] / dTb[0] : 0.0;
  out[9] = (s.nf == 4) ? dT[1] / dTb[1] : 0.0;
  out[10] = dvmax;
  out[11] = sqrt(dv2 / vol);
  out[12] = sc->rate_last * sc->dt;
}

}  // namespace

void launch_diagnostics(tc_ctx *c) {
  const Sizes &s = c->sz;
  Radial rad = c->nl.rad;
  LaunchScope ls(c, KDIAG);
  k_diag_level<<<s.Nr, kDiagThreads, 0, c->stream>>>(c->X, c->base_dev, c->diag_part, s, rad,
                                                     c->nl.alpha);
  double *Tb = c->diag_part + s.Nr * kNPart;
  c->launches++;
  k_diag_final<<<1, 1, 0, c->stream>>>(c->X, c->diag_part, Tb, c->diag_out, s, rad,
                                       2.0 * 3.14159265358979323846 * c->Lz, c->Gr, c->Re_i,
                                       c->Re_o, c->scal);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// FP64 FMA rate of the device, for the ALU roofline of the FP64 kernels.
// Every thread runs 4 independent dependent chains x <- fma(x, a, b) (a, b
// kernel arguments, so nothing folds), 32 warps on every SM: the FP64 unit
// of every SM sub-partition is kept busy whatever its latency.
namespace tc {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 4;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_rate(double *out, int iters, double a,
                                                              double b) {
  double x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_measure_fp64_rate(double target_ms, void *stream, double *tflops) {
  if (!tflops || !(target_ms > 0.0) || target_ms > 10000.0) return TC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return TC_ERR_CUDA;
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)nsm * tc::kProbeThreads) != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double total_ms = 0.0, total_flops = 0.0;
  // one calibration launch, then launches of about a tenth of the target each
  int iters = 4000;
  const double a = 0.999999, b = 1e-7;
  for (int rep = 0; e == cudaSuccess && rep < 12 && total_ms < target_ms; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) break;
    tc::k_fp64_rate<<<nsm, tc::kProbeThreads, 0, st>>>(buf, iters, a, b);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess || ms <= 0.0f) break;
    if (rep > 0) {   // the calibration launch also settles the clock
      total_ms += ms;
      total_flops += 2.0 * tc::kProbeChains * (double)iters * nsm * tc::kProbeThreads;
    }
    const double want = target_ms / 10.0;
    const double next = iters * want / ms;
    iters = (int)std::min(4.0e5, std::max(1000.0, next));   // at most ~0.5 s per launch
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_CUDA;
  }
  if (total_ms <= 0.0) return TC_ERR_CUDA;
  *tflops = total_flops / (total_ms * 1e-3) / 1e12;
  return TC_OK;
}
