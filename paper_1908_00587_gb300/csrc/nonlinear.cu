// Nonlinear stage: dealiased u.grad u (and u.grad T) on the 3/2 grid.
//
// Paper Sec. 2.1/2.2: the nonlinear terms are formed pseudospectrally, after
// gathering all Fourier modes of a radial level (the MPI code transposes
// between mode slabs and radial slabs; here every radial level is already
// resident on the one GPU, so the "transpose" is only the choice of which
// index a CTA walks).  Three kernels per evaluation:
//   k_zinv   per (m-block, r, component): fill the padded axial spectrum of
//            the value, its radial derivative (9-point stencil) and its axial
//            derivative (i beta), inverse FFT along z.  The theta derivative
//            is formed later as i m times the value's z-transform.
//   k_theta  per (z-row block, r): inverse FFT along theta of 2 real fields per
//            complex transform, pointwise products with the curvature terms
//            and buoyancy, CFL rate, forward FFT along theta, keep m <= M.
//   k_zfwd   per (m-block, r): forward FFT along z, keep |k| <= K, scale.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "fft.cuh"
#include "nl_body.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

__global__ void k_meanprof(const double2 *__restrict__ X, double *__restrict__ prof,
                           float *__restrict__ prof32, Sizes s, Radial rad) {
  meanprof_body(X, prof, prof32, s, rad, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_tofloat(const double2 *__restrict__ X, float2 *__restrict__ X32, Sizes s) {
  tofloat_body(X, X32, s, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void k_zinv(const V2<T> *__restrict__ X, V2<T> *__restrict__ Vout, NLParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zinv_body<T>(X, Vout, p, smem_raw, blockIdx.x, blockIdx.y, blockIdx.z);
}

// mode 0: nonlinear products -> W; mode 1: max |u| and max |T| (initial state scaling)
template <typename T>
__global__ void k_theta(const V2<T> *__restrict__ Vin, V2<T> *__restrict__ W, NLParams p,
                        unsigned long long *__restrict__ rate_bits,
                        unsigned long long *__restrict__ norm_bits, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  theta_body<T>(Vin, W, p, rate_bits, norm_bits, mode, smem_raw, blockIdx.x, blockIdx.y);
}

// W layout [g][r][l][m] -> N [g][r][m][kk]
template <typename T>
__global__ void k_zfwd(const V2<T> *__restrict__ W, double2 *__restrict__ N, NLParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zfwd_body<T>(W, N, p, smem_raw, blockIdx.x, blockIdx.y);
}

}  // namespace

unsigned debug_word_nonlinear(int clear) {
  unsigned v = 0;
#ifdef TC_DEBUG
  if (cudaMemcpyFromSymbol(&v, g_dbg_word, sizeof(v)) != cudaSuccess) cudaGetLastError();
  if (clear) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_dbg_word, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
  }
#else
  (void)clear;
#endif
  return v;
}

void set_divisors(NLParams &p) {
  const Sizes &s = p.sz;
  p.fNK = make_fastdiv((unsigned)s.NK);
  p.fNM = make_fastdiv((unsigned)s.NM);
  p.fNt = make_fastdiv((unsigned)s.Nt);
  p.fNz = make_fastdiv((unsigned)s.Nz);
  p.fnf = make_fastdiv((unsigned)s.nf);
  p.fMB = make_fastdiv((unsigned)p.MB);
  const int last = s.NM - ((s.NM - 1) / p.MB) * p.MB;   // width of the last m-block
  p.fMBl = make_fastdiv((unsigned)last);
  p.fMBf = make_fastdiv((unsigned)p.MBf);
  const int lastf = s.NM - ((s.NM - 1) / p.MBf) * p.MBf;
  p.fMBfl = make_fastdiv((unsigned)lastf);
}

void setup_nonlinear(tc_ctx *c) {
  NLParams &p = c->nl;
  const Sizes &s = c->sz;
  const size_t e = sizeof(double2);
  // z kernels: at most ~48 KB per ping-pong buffer
  int MB = (int)(3072 / (3 * s.Nz));
  if (MB < 1) MB = 1;
  if (MB > 8) MB = 8;
  if (c->tile_mb > 0) MB = c->tile_mb;
  if (MB > s.NM) MB = s.NM;
  p.MB = MB;
  p.MBf = (c->tile_mbf > 0) ? std::min(c->tile_mbf, s.NM) : MB;
  int LB = (int)(4096 / (2 * s.nf * s.Nt));
  if (LB < 1) LB = 1;
  if (LB > 8) LB = 8;
  if (c->tile_lb > 0) LB = c->tile_lb;
  p.LB = LB;
  c->smem_zinv = (size_t)(2 * 3 * MB * padlen(s.Nz) + s.Nz) * e;
  c->smem_theta = (size_t)(2 * LB * 2 * s.nf * padlen(s.Nt) + s.Nt) * e;
  c->smem_zfwd = (size_t)(2 * s.nf * p.MBf * padlen(s.Nz) + s.Nz) * e;
  allow_smem(k_zinv<double>);
  allow_smem(k_theta<double>);
  allow_smem(k_zfwd<double>);
  // FP32 copies of the transforms (mixed precision): same blocking by bytes
  NLParams &q = c->nl32;
  q = p;
  const size_t e32 = sizeof(float2);
  int MB32 = (int)(6144 / (3 * s.Nz));
  MB32 = MB32 < 1 ? 1 : (MB32 > 8 ? 8 : MB32);
  if (c->tile_mb > 0) MB32 = c->tile_mb;
  if (MB32 > s.NM) MB32 = s.NM;
  int LB32 = (int)(8192 / (2 * s.nf * s.Nt));
  LB32 = LB32 < 1 ? 1 : (LB32 > 8 ? 8 : LB32);
  if (c->tile_lb > 0) LB32 = c->tile_lb;
  q.MB = MB32;
  q.MBf = (c->tile_mbf > 0) ? std::min(c->tile_mbf, s.NM) : MB32;
  q.LB = LB32;
  set_divisors(p);
  set_divisors(q);
  c->smem32_zinv = (size_t)(2 * 3 * MB32 * padlen(s.Nz) + s.Nz) * e32;
  c->smem32_theta = (size_t)(2 * LB32 * 2 * s.nf * padlen(s.Nt) + s.Nt) * e32;
  c->smem32_zfwd = (size_t)(2 * s.nf * q.MBf * padlen(s.Nz) + s.Nz) * e32;
  allow_smem(k_zinv<float>);
  allow_smem(k_theta<float>);
  allow_smem(k_zfwd<float>);
}

void launch_nonlinear(tc_ctx *c, const double2 *X, double2 *N, unsigned long long *rate_bits,
                      int mode, double2 *phys_out) {
  const Sizes &s = c->sz;
  if (c->precision == 1 && mode == 0) {
    NLParams q = c->nl32;
    q.mixed = 1;
    q.Xfull = X;
    q.prof = c->prof;
    float2 *V = reinterpret_cast<float2 *>(c->V);
    float2 *W = reinterpret_cast<float2 *>(c->W);
    {
      LaunchScope ls(c, KZINV);
      k_meanprof<<<(s.Nr + 63) / 64, 64, 0, c->stream>>>(X, c->prof, c->d_prof32, s, q.rad);
      k_tofloat<<<(unsigned)(((long long)s.nf * s.S + 255) / 256), 256, 0, c->stream>>>(
          X, c->X32, s);
      k_zinv<float><<<dim3((s.NM + q.MB - 1) / q.MB, s.Nr, s.nf), 256, c->smem32_zinv,
                      c->stream>>>(c->X32, V, q);
    }
    {
      LaunchScope ls(c, KTHETA);
      k_theta<float><<<dim3((s.Nz + q.LB - 1) / q.LB, s.Nr), 256, c->smem32_theta,
                       c->stream>>>(V, W, q, rate_bits, c->scal->norm_bits, 0);
    }
    LaunchScope ls(c, KZFWD);
    k_zfwd<float><<<dim3((s.NM + q.MBf - 1) / q.MBf, s.Nr), 256, c->smem32_zfwd, c->stream>>>(
        W, N, q);
    return;
  }
  NLParams p = c->nl;
  p.phys_out = phys_out;
  const int nmb = (s.NM + p.MB - 1) / p.MB;
  if (mode == 0 && !phys_out && c->tensor_z && c->d_dft_ztc) {
    LaunchScope ls(c, KZINVTC);
    launch_zinv_tc(c->stream, X, c->V, p, c->d_dft_ztc, &c->scal->timeout, !c->selftest_no_copy);
  } else {
    LaunchScope ls(c, KZINV);
    k_zinv<double><<<dim3(nmb, s.Nr, s.nf), 256, c->smem_zinv, c->stream>>>(X, c->V, p);
  }
  const int nlb = (s.Nz + p.LB - 1) / p.LB;
  alignas(64) unsigned char vmap[128];
  if (mode == 0 && !phys_out && c->tensor_theta && c->d_dft_tc && theta_tc_map(vmap, c->V, s)) {
    LaunchScope ls(c, KTHETATC);
    launch_theta_tc(c->stream, vmap, c->W, p, c->d_dft_tc, rate_bits, &c->scal->timeout,
                    !c->selftest_no_copy);
  } else {
    LaunchScope ls(c, KTHETA);
    k_theta<double><<<dim3(nlb, s.Nr), 256, c->smem_theta, c->stream>>>(
        c->V, c->W, p, rate_bits, c->scal->norm_bits, mode);
  }
  if (mode == 1) return;
  LaunchScope ls(c, KZFWD);
  k_zfwd<double><<<dim3((s.NM + p.MBf - 1) / p.MBf, s.Nr), 256, c->smem_zfwd, c->stream>>>(
      c->W, N, p);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Allocation-free nonlinear stage (tc_nonlinear_noalloc in include/tc.h).
//
// Same three kernels as launch_nonlinear, but every buffer beyond the caller's
// input and output -- radial tables, twiddles, the z- and theta-transformed
// intermediates and the CFL slot -- lives in one file-scope device array of
// kNoAllocBytes.  Every GPU that loads this library holds that array until
// the process exits.  All calls share it: a call overwrites whatever the last
// call left there (the CFL slot is cleared each call; the tables and both
// intermediates are written in full before they are read), and calls that
// overlap on the GPU race on it.
namespace tc {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB
constexpr int kNoAllocMaxNr = 256;
constexpr int kNoAllocMaxN = 512;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
// device address of the array per device, looked up once per device; atomic
// so that host threads calling at the same time do not race (they would
// store the same address)
std::atomic<unsigned char *> g_scratch_addr[kMaxDevices] = {};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the pieces inside the scratch array.
struct NoAllocLayout {
  size_t r, inv_r, dr, cinv, D1, s0, twz, twt, rate, table_end, V, W, end;
};

NoAllocLayout noalloc_layout(const Sizes &s) {
  NoAllocLayout L{};
  size_t o = 0;
  L.r = o;      o = align256(o + sizeof(double) * s.Nr);
  L.inv_r = o;  o = align256(o + sizeof(double) * s.Nr);
  L.dr = o;     o = align256(o + sizeof(double) * s.Nr);
  L.cinv = o;   o = align256(o + sizeof(double) * 2 * s.Nr);
  L.D1 = o;     o = align256(o + sizeof(double) * s.Nr * kStencil);
  L.s0 = o;     o = align256(o + sizeof(int) * s.Nr);
  L.twz = o;    o = align256(o + sizeof(double2) * s.Nz);
  L.twt = o;    o = align256(o + sizeof(double2) * s.Nt);
  L.rate = o;   o = align256(o + sizeof(unsigned long long));
  L.table_end = o;
  const size_t plane = sizeof(double2) * (size_t)s.Nr * s.Nz * s.NM;
  L.V = o;      o = align256(o + plane * 3 * s.nf);
  L.W = o;      o = align256(o + plane * s.nf);
  L.end = o;
  return L;
}

// Largest table segment a call can need (host staging block on the stack).
constexpr size_t kTableMaxBytes =
    3 * (kNoAllocMaxNr * 8 + 256) + (2 * kNoAllocMaxNr * 8 + 256) +
    (kNoAllocMaxNr * kStencil * 8 + 256) +
    (kNoAllocMaxNr * 4 + 256) + 2 * (kNoAllocMaxN * 16 + 256) + 256;

bool smooth235_na(int n) {
  if (n < 1) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_nonlinear_noalloc(int Nr, int Ntheta, int Nz, double eta, double Lz,
                                          double Ra, double Pr, const void *state_dev,
                                          void *n_dev, void *stream, double *cfl_rate) {
  using namespace tc;
  if (!state_dev || !n_dev) return TC_ERR_ARG;
  if (Nr < kStencil || Ntheta < 4 || Ntheta % 2 != 0 || Nz < 4) return TC_ERR_ARG;
  if (!smooth235_na(Ntheta) || !smooth235_na(Nz)) return TC_ERR_ARG;
  if (!(eta > 0.0 && eta < 1.0) || !(Lz > 0.0) || !std::isfinite(Lz) || !std::isfinite(Ra))
    return TC_ERR_ARG;
  if (Ra != 0.0 && !(Pr > 0.0 && std::isfinite(Pr))) return TC_ERR_ARG;
  // size limit of the static scratch: reject with TC_ERR_UNSUPPORTED
  if (Nr > kNoAllocMaxNr || Ntheta > kNoAllocMaxN || Nz > kNoAllocMaxN) return TC_ERR_UNSUPPORTED;
  Sizes s{};
  s.Nr = Nr;
  s.Nt = Ntheta;
  s.Nz = Nz;
  s.M = (Ntheta - 1) / 3;
  s.K = (Nz - 1) / 3;
  s.NM = s.M + 1;
  s.NK = 2 * s.K + 1;
  s.nmode = s.NM * s.NK;
  s.nf = (Ra != 0.0) ? 4 : 3;
  s.S = (long long)Nr * s.nmode;
  const NoAllocLayout L = noalloc_layout(s);
  if (L.end > kNoAllocBytes) return TC_ERR_UNSUPPORTED;

  // launch geometry: the same rules as the context path
  NLParams p{};
  p.sz = s;
  int MB = (int)(3072 / (3 * s.Nz));
  MB = MB < 1 ? 1 : (MB > 8 ? 8 : MB);
  if (MB > s.NM) MB = s.NM;
  int LB = (int)(4096 / (2 * s.nf * s.Nt));
  LB = LB < 1 ? 1 : (LB > 8 ? 8 : LB);
  p.MB = MB;
  p.MBf = MB;
  p.LB = LB;
  set_divisors(p);
  const size_t e = sizeof(double2);
  const size_t sm_zinv = (size_t)(2 * 3 * MB * padlen(s.Nz) + s.Nz) * e;
  const size_t sm_theta = (size_t)(2 * LB * 2 * s.nf * padlen(s.Nt) + s.Nt) * e;
  const size_t sm_zfwd = (size_t)(2 * s.nf * MB * padlen(s.Nz) + s.Nz) * e;
  if (sm_zinv > 227 * 1024 || sm_theta > 227 * 1024 || sm_zfwd > 227 * 1024)
    return TC_ERR_UNSUPPORTED;

  // once per device, with that device current: the device address of the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TC_ERR_CUDA;
  unsigned char *base = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
    base = static_cast<unsigned char *>(ptr);
    g_scratch_addr[dev].store(base, std::memory_order_release);
  }

  // radial tables and twiddles, staged on the host stack and copied in
  alignas(256) unsigned char host[kTableMaxBytes];
  const double r_i = eta / (1.0 - eta);
  double *r = reinterpret_cast<double *>(host + L.r);
  double *inv_r = reinterpret_cast<double *>(host + L.inv_r);
  double *drm = reinterpret_cast<double *>(host + L.dr);
  double *cinv = reinterpret_cast<double *>(host + L.cinv);
  double *D1 = reinterpret_cast<double *>(host + L.D1);
  int *s0 = reinterpret_cast<int *>(host + L.s0);
  for (int j = 0; j < Nr; ++j) {
    r[j] = r_i + 0.5 * (1.0 - std::cos(M_PI * (double)j / (double)(Nr - 1)));
    inv_r[j] = 1.0 / r[j];
  }
  for (int j = 0; j < Nr; ++j) {
    const int st = std::min(std::max(j - kStencil / 2, 0), Nr - kStencil);
    s0[j] = st;
    double w[3][kStencil];
    fd_weights(r[j], &r[st], kStencil, w);
    for (int t = 0; t < kStencil; ++t) D1[j * kStencil + t] = w[1][t];
    const double lo = j > 0 ? r[j] - r[j - 1] : 1e300;
    const double hi = j < Nr - 1 ? r[j + 1] - r[j] : 1e300;
    drm[j] = std::min(lo, hi);
    cinv[2 * j] = 1.0 / drm[j];
    cinv[2 * j + 1] = 1.0 / (r[j] * (2.0 * M_PI / Ntheta));
  }
  fill_plan_twiddles(make_plan(Nz), reinterpret_cast<double2 *>(host + L.twz));
  fill_plan_twiddles(make_plan(Ntheta), reinterpret_cast<double2 *>(host + L.twt));
  *reinterpret_cast<unsigned long long *>(host + L.rate) = 0ull;   // CFL slot starts at zero

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(base, host, L.table_end, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_CUDA;
  }
  p.rad = Radial{reinterpret_cast<const double *>(base + L.r),
                 reinterpret_cast<const double *>(base + L.inv_r),
                 reinterpret_cast<const double *>(base + L.D1), nullptr,
                 reinterpret_cast<const double *>(base + L.dr), nullptr,
                 reinterpret_cast<const int *>(base + L.s0)};
  p.alpha = 2.0 * M_PI / Lz;
  p.Gr = (Ra != 0.0) ? Ra / Pr : 0.0;
  p.dth = 2.0 * M_PI / s.Nt;
  p.dz = Lz / s.Nz;
  p.inv_dz = 1.0 / p.dz;
  p.cfl_inv = reinterpret_cast<const double *>(base + L.cinv);
  p.zscale = 0.5 / ((double)s.Nt * (double)s.Nz);
  p.pz = make_plan(s.Nz);
  p.pt = make_plan(s.Nt);
  p.twz = reinterpret_cast<const double2 *>(base + L.twz);
  p.twt = reinterpret_cast<const double2 *>(base + L.twt);
  double2 *V = reinterpret_cast<double2 *>(base + L.V);
  double2 *W = reinterpret_cast<double2 *>(base + L.W);
  unsigned long long *rate = reinterpret_cast<unsigned long long *>(base + L.rate);

  allow_smem(k_zinv<double>);
  allow_smem(k_theta<double>);
  allow_smem(k_zfwd<double>);
  const int nmb = (s.NM + MB - 1) / MB;
  const int nlb = (s.Nz + LB - 1) / LB;
  k_zinv<double><<<dim3(nmb, s.Nr, s.nf), 256, sm_zinv, st>>>(
      static_cast<const double2 *>(state_dev), V, p);
  k_theta<double><<<dim3(nlb, s.Nr), 256, sm_theta, st>>>(V, W, p, rate, nullptr, 0);
  k_zfwd<double><<<dim3(nmb, s.Nr), 256, sm_zfwd, st>>>(W, static_cast<double2 *>(n_dev), p);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (cfl_rate) {
    unsigned long long bits = 0;
    if (cudaMemcpyAsync(&bits, rate, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
    std::memcpy(cfl_rate, &bits, sizeof(double));
  }
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Adjoint of the nonlinear stage (FP64): Nbar (primitive cotangents of N) ->
// Xbar += (dN/dX)^T Nbar at the linearisation point X, in the real Euclidean
// inner product of stored (Re, Im) coefficients.
//   * adjoint of the forward transform (scaled by 1/(Ntheta Nz)) is
//     1/(Ntheta Nz) times the inverse transform of the cotangent with the
//     m >= 1 entries halved;
//   * adjoint of the pointwise products (linearised about X's fields);
//   * adjoint of the inverse transform is the unnormalised forward transform
//     with the m >= 1 entries doubled; derivative multipliers i m, i beta
//     become -i m, -i beta, and d/dr becomes the transposed stencil.
namespace tc {
namespace {

// z-inverse of the cotangent (values only, m >= 1 halved): V2 [nf][r][l][m]
__global__ void k_zinv_adj(const double2 *__restrict__ Nb, double2 *__restrict__ Vout,
                           NLParams p) {
  const Sizes &s = p.sz;
  const int m0 = blockIdx.x * p.MB;
  const int nm = min(p.MB, s.NM - m0);
  const int r = blockIdx.y;
  const int Nz = s.Nz;
  const int Np = padlen(Nz);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);
  double2 *B = A + s.nf * p.MB * Np;
  double2 *tw = B + s.nf * p.MB * Np;
  load_tw<double>(tw, p.twz, nullptr, Nz);
  for (int i = threadIdx.x; i < s.nf * nm * Np; i += blockDim.x) A[i] = double2{0, 0};
  __syncthreads();
  for (int t = threadIdx.x; t < s.nf * nm * s.NK; t += blockDim.x) {
    const int kk = t % s.NK;
    const int rest = t / s.NK;
    const int mi = rest % nm;
    const int g = rest / nm;
    const int m = m0 + mi;
    const double h = (m == 0) ? 1.0 : 0.5;
    const double2 v = Nb[(long long)g * s.S + (long long)r * s.nmode + (long long)m * s.NK + kk];
    A[(g * nm + mi) * Np + spad(kpos(kk, s.K, s.NK, Nz))] = double2{h * v.x, h * v.y};
  }
  __syncthreads();
  double2 *res = fft_batch<+1>(A, B, p.pz, s.nf * nm, Np, tw);
  for (int t = threadIdx.x; t < s.nf * nm * Nz; t += blockDim.x) {
    const int mi = t % nm;
    const int rest = t / nm;
    const int l = rest % Nz;
    const int g = rest / Nz;
    Vout[(((long long)g * s.Nr + r) * Nz + l) * s.NM + m0 + mi] = res[(g * nm + mi) * Np + spad(l)];
  }
}

// Per z-row: forward fields of X (from V) and the cotangent (from V2) to the
// physical grid, pointwise adjoint of the products, forward theta-transform of
// the 4 nf field cotangents.  Output Wa [3c + d][r][l][m], d = 0: value with
// the theta part folded in (c'_m (G_val - i m G_theta)), 1: d/dr, 2: d/dz.
__global__ void k_theta_adj(const double2 *__restrict__ Vin, const double2 *__restrict__ V2,
                            double2 *__restrict__ Wa, NLParams p) {
  const Sizes &s = p.sz;
  const int l0 = blockIdx.x * p.LB;
  const int nl = min(p.LB, s.Nz - l0);
  const int r = blockIdx.y;
  const int Nt = s.Nt;
  const int Ntp = padlen(Nt);
  const int nfw = 2 * s.nf;          // forward-field pairs per row
  // transformed here per row: the forward pairs (unless phys_in holds them)
  // and the cotangent pairs (N_r, N_theta), (N_z, N_T)
  const bool cached = p.phys_in != nullptr;
  const int npair = cached ? 2 : nfw + 2;
  const int cot0 = cached ? 0 : nfw;   // first cotangent pair of a row
  const int nbuf = p.LB * (nfw + 2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);
  double2 *B = A + nbuf * Ntp;
  double2 *tw = B + nbuf * Ntp;
  load_tw<double>(tw, p.twt, nullptr, Nt);
  for (int i = threadIdx.x; i < nl * npair * Ntp; i += blockDim.x) A[i] = double2{0, 0};
  __syncthreads();
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  const int nin = cached ? 2 : s.nf + 2;   // inputs per row: components, then 2 cotangent pairs
  for (int t = threadIdx.x; t < nl * nin * s.NM; t += blockDim.x) {
    const int2 q1 = divmod(t, s.NM, p.fNM);
    const int m = q1.y;
    const int li = q1.x / nin;
    const int c = q1.x - li * nin + (cached ? s.nf : 0);
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    double2 a, b, e, f;
    double2 *b0, *b1;
    if (c < s.nf) {
      a = Vin[(3 * c + 0) * fs + off];
      e = Vin[(3 * c + 1) * fs + off];
      f = Vin[(3 * c + 2) * fs + off];
      if (m == 0) {
        a.y = 0.0;
        e.y = 0.0;
        f.y = 0.0;
      }
      b = double2{-(double)m * a.y, (double)m * a.x};   // i m a
      b0 = A + (li * npair + 2 * c) * Ntp;
      b1 = b0 + Ntp;
    } else {
      const int h = c - s.nf;   // 0: (N_r, N_theta), 1: (N_z, N_T)
      a = V2[(2 * h) * fs + off];
      b = (2 * h + 1 < s.nf) ? V2[(2 * h + 1) * fs + off] : double2{0.0, 0.0};
      if (m == 0) {
        a.y = 0.0;
        b.y = 0.0;
      }
      b0 = A + (li * npair + cot0 + h) * Ntp;
      b1 = nullptr;
    }
    b0[spad(m)] = double2{a.x - b.y, a.y + b.x};
    if (m > 0) b0[spad(Nt - m)] = double2{a.x + b.y, -a.y + b.x};
    if (b1) {
      b1[spad(m)] = double2{e.x - f.y, e.y + f.x};
      if (m > 0) b1[spad(Nt - m)] = double2{e.x + f.y, -e.y + f.x};
    }
  }
  __syncthreads();
  double2 *ph = fft_batch<+1>(A, B, p.pt, nl * npair, Ntp, tw);
  double2 *out = (ph == A) ? B : A;
  const double ir = p.rad.inv_r[r];
  const double sc = 1.0 / ((double)s.Nt * (double)s.Nz);
  for (int t = threadIdx.x; t < nl * Nt; t += blockDim.x) {
    const int2 a = divmod(t, Nt, p.fNt);
    const int j = a.y;
    const int li = a.x;
    const double2 *b = ph + li * npair * Ntp + spad(j);
    // forward pairs: from this kernel's transforms, or the stored physical fields
    const double2 *f = cached ? p.phys_in + ((long long)r * s.Nz + l0 + li) * nfw * Nt + j : b;
    const int fst = cached ? Nt : Ntp;
    const double2 r0 = f[0 * fst], r1 = f[1 * fst];   // (ur, ur_t), (ur_r, ur_z)
    const double2 t0 = f[2 * fst], t1 = f[3 * fst];
    const double2 z0 = f[4 * fst], z1 = f[5 * fst];
    const double2 nb0 = b[cot0 * Ntp], nb1 = b[(cot0 + 1) * Ntp];
    const double ar = sc * nb0.x, at = sc * nb0.y, az = sc * nb1.x, aT = sc * nb1.y;
    const double ur = r0.x, ut = t0.x, uz = z0.x;
    const double vt = ut * ir;
    // cotangents of the 4 nf physical input fields
    double gur = -(r1.x * ar) - (t1.x + vt) * at - z1.x * az;
    double gut = -(r0.y * ir) * ar + 2.0 * vt * ar - (t0.y * ir) * at - (ur * ir) * at -
                 (z0.y * ir) * az;
    double guz = -(r1.y * ar) - t1.y * at - z1.y * az;
    const double gurr = -ur * ar, gurt = -vt * ar, gurz = -uz * ar;
    const double gutr = -ur * at, gutt = -vt * at, gutz = -uz * at;
    const double guzr = -ur * az, guzt = -vt * az, guzz = -uz * az;
    double gT = 0.0, gTr = 0.0, gTt = 0.0, gTz = 0.0;
    if (s.nf == 4) {
      const double2 T0 = f[6 * fst], T1 = f[7 * fst];
      gur -= T1.x * aT;
      gut -= (T0.y * ir) * aT;
      guz -= T1.y * aT;
      gT = p.Gr * az;
      gTr = -ur * aT;
      gTt = -vt * aT;
      gTz = -uz * aT;
    }
    double2 *o = out + li * nfw * Ntp + spad(j);
    o[0 * Ntp] = double2{gur, gurt};
    o[1 * Ntp] = double2{gurr, gurz};
    o[2 * Ntp] = double2{gut, gutt};
    o[3 * Ntp] = double2{gutr, gutz};
    o[4 * Ntp] = double2{guz, guzt};
    o[5 * Ntp] = double2{guzr, guzz};
    if (s.nf == 4) {
      o[6 * Ntp] = double2{gT, gTt};
      o[7 * Ntp] = double2{gTr, gTz};
    }
  }
  __syncthreads();
  double2 *scratch = (out == A) ? B : A;
  double2 *sp = fft_batch<-1>(out, scratch, p.pt, nl * nfw, Ntp, tw);
  for (int t = threadIdx.x; t < nl * s.nf * s.NM; t += blockDim.x) {
    const int2 q1 = divmod(t, s.NM, p.fNM);
    const int m = q1.y;
    const int2 q2 = divmod(q1.x, s.nf, p.fnf);
    const int c = q2.y;
    const int li = q2.x;
    const double cm = (m == 0) ? 1.0 : 2.0;
    const int mm = (Nt - m) % Nt;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const double2 *z0 = sp + (li * nfw + 2 * c) * Ntp;
    // pair (val, theta): X = value part, Y = theta part
    const double2 a = z0[spad(m)], bq = z0[spad(mm)];
    const double2 Gv = double2{0.5 * (a.x + bq.x), 0.5 * (a.y - bq.y)};
    const double2 Gt = double2{0.5 * (a.y + bq.y), 0.5 * (bq.x - a.x)};
    // value cotangent with the theta derivative folded in: c'_m (Gv - i m Gt)
    Wa[(3 * c + 0) * fs + off] = double2{cm * (Gv.x + m * Gt.y), cm * (Gv.y - m * Gt.x)};
    const double2 *z1 = z0 + Ntp;
    const double2 a1 = z1[spad(m)], b1 = z1[spad(mm)];
    const double2 Gr = double2{0.5 * (a1.x + b1.x), 0.5 * (a1.y - b1.y)};
    const double2 Gz = double2{0.5 * (a1.y + b1.y), 0.5 * (b1.x - a1.x)};
    Wa[(3 * c + 1) * fs + off] = double2{cm * Gr.x, cm * Gr.y};
    Wa[(3 * c + 2) * fs + off] = double2{cm * Gz.x, cm * Gz.y};
  }
}

// z-forward (unnormalised) of Wa; Xb += val - i beta z-part; Gr [c][r][mode]
// holds the d/dr cotangent for the transposed stencil.
__global__ void k_zfwd_adj(const double2 *__restrict__ Wa, double2 *__restrict__ Xb,
                           double2 *__restrict__ Gr, NLParams p, int accumulate) {
  const Sizes &s = p.sz;
  const int m0 = blockIdx.x * p.MB;
  const int nm = min(p.MB, s.NM - m0);
  const int r = blockIdx.y;
  const int c = blockIdx.z;
  const int Nz = s.Nz;
  const int Np = padlen(Nz);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);
  double2 *B = A + 3 * p.MB * Np;
  double2 *tw = B + 3 * p.MB * Np;
  load_tw<double>(tw, p.twz, nullptr, Nz);
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  for (int t = threadIdx.x; t < 3 * nm * Nz; t += blockDim.x) {
    const int mi = t % nm;
    const int rest = t / nm;
    const int l = rest % Nz;
    const int d = rest / Nz;
    A[(3 * mi + d) * Np + spad(l)] = Wa[(3 * c + d) * fs + ((long long)r * Nz + l) * s.NM + m0 + mi];
  }
  __syncthreads();
  double2 *res = fft_batch<-1>(A, B, p.pz, 3 * nm, Np, tw);
  for (int t = threadIdx.x; t < nm * s.NK; t += blockDim.x) {
    const int kk = t % s.NK;
    const int mi = t / s.NK;
    const int pos = spad(kpos(kk, s.K, s.NK, Nz));
    const double beta = p.betak[kk];   // alpha k (FP64 table: no conversion on the FP64 unit)
    const double2 v = res[(3 * mi + 0) * Np + pos];
    const double2 gr = res[(3 * mi + 1) * Np + pos];
    const double2 gz = res[(3 * mi + 2) * Np + pos];
    const long long i = (long long)c * s.S + (long long)r * s.nmode + (long long)(m0 + mi) * s.NK + kk;
    double2 x = double2{v.x + beta * gz.y, v.y - beta * gz.x};   // v - i beta gz
    if (accumulate) {
      const double2 o = Xb[i];
      x.x += o.x;
      x.y += o.y;
    }
    Xb[i] = x;
    Gr[i] = gr;
  }
}

// Xb(s) += sum_j D1[j][s - s0_j] Gr(j)  (transposed radial stencil)
__global__ void k_drT(const double2 *__restrict__ Gr, double2 *__restrict__ Xb, Sizes s,
                      Radial rad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)s.nf * s.S) return;
  const int c = (int)(i / s.S);
  const long long rem = i - (long long)c * s.S;
  const int sn = (int)(rem / s.nmode);
  const int mode = (int)(rem - (long long)sn * s.nmode);
  double2 acc = Xb[i];
  for (int e = 0; e < kTrans; ++e) {
    const int j = rad.tj[sn * kTrans + e];
    if (j < 0) break;
    const int t = sn - rad.s0[j];
    const double w = rad.D1[j * kStencil + t];
    const double2 g = Gr[(long long)c * s.S + (long long)j * s.nmode + mode];
    acc.x += w * g.x;
    acc.y += w * g.y;
  }
  Xb[i] = acc;
}

}  // namespace

// The adjoint's azimuthal kernel holds 2 nf + 2 sequences per z-row, so it
// takes the largest z-row tile not above the forward one that fits.
// Tiles of the adjoint's nonlinear kernels: the largest not above the forward
// ones (at most 4 m-columns) whose shared memory lets three CTAs share an SM,
// so that small runs still spread over every SM (the forward tiles are tuned
// for the forward kernels, whose buffers are smaller).  4 m-columns give the
// axial kernels' first radix-8 pass 3 x 4 x Nz/8 butterflies, whole warps at
// Nz = 64 (with 2, a warp in two runs half empty, and a warp's FP64
// instruction costs the same however many lanes are active): the adjoint
// step at 64^3 1.084 -> 1.054 ms, the recorded one 0.612 -> 0.589 ms.
static const size_t kAdjSmemPerCta = (size_t)74 * 1024;
static size_t adj_theta_smem(const Sizes &s, int lb) {
  return (size_t)(2 * lb * (2 * s.nf + 2) * padlen(s.Nt) + s.Nt) * sizeof(double2);
}
static size_t adj_z_smem(const Sizes &s, int mb) {   // the larger of k_zinv_adj, k_zfwd_adj, k_zinv
  const int w = s.nf > 3 ? s.nf : 3;
  return (size_t)(2 * w * mb * padlen(s.Nz) + s.Nz) * sizeof(double2);
}
static int adjoint_lb(const tc_ctx *c) {
  int lb = c->nl.LB;
  while (lb > 1 && adj_theta_smem(c->sz, lb) > kAdjSmemPerCta) --lb;
  return lb;
}
static int adjoint_mb(const tc_ctx *c) {
  int mb = c->nl.MB < 4 ? c->nl.MB : 4;
  if (c->tile_mb_adj > 0) mb = std::min(c->tile_mb_adj, c->sz.NM);
  while (mb > 1 && adj_z_smem(c->sz, mb) > kAdjSmemPerCta) --mb;
  return mb;
}

void setup_nonlinear_adjoint(tc_ctx *c) {
  (void)c;
  allow_smem(k_zinv_adj);
  allow_smem(k_theta_adj);
  allow_smem(k_zfwd_adj);
}

void launch_nonlinear_adjoint(tc_ctx *c, const double2 *X, const double2 *Nb, double2 *Xb,
                              int accumulate, const double2 *phys_in) {
  const Sizes &s = c->sz;
  NLParams p = c->nl;
  p.LB = adjoint_lb(c);
  p.MB = adjoint_mb(c);
  set_divisors(p);
  p.phys_in = phys_in;
  const size_t e = sizeof(double2);
  c->smem_adj_zinv = (size_t)(2 * s.nf * p.MB * padlen(s.Nz) + s.Nz) * e;
  c->smem_adj_theta = adj_theta_smem(s, p.LB);
  c->smem_adj_zfwd = (size_t)(2 * 3 * p.MB * padlen(s.Nz) + s.Nz) * e;
  const size_t smem_zinv = (size_t)(2 * 3 * p.MB * padlen(s.Nz) + s.Nz) * e;
  const int nmb = (s.NM + p.MB - 1) / p.MB;
  const int nlb = (s.Nz + p.LB - 1) / p.LB;
  if (!phys_in) {   // the forward fields of X, unless stored by the forward pass
    LaunchScope ls(c, KZINV);
    k_zinv<double><<<dim3(nmb, s.Nr, s.nf), 256, smem_zinv, c->stream>>>(X, c->V, p);
  }
  {
    LaunchScope ls(c, KZINV);
    k_zinv_adj<<<dim3(nmb, s.Nr), 256, c->smem_adj_zinv, c->stream>>>(Nb, c->W, p);
  }
  {
    LaunchScope ls(c, KTHETA);
    k_theta_adj<<<dim3(nlb, s.Nr), 256, c->smem_adj_theta, c->stream>>>(c->V, c->W, c->Va, p);
  }
  {
    LaunchScope ls(c, KZFWD);
    k_zfwd_adj<<<dim3(nmb, s.Nr, s.nf), 256, c->smem_adj_zfwd, c->stream>>>(c->Va, Xb, c->Gdr,
                                                                            p, accumulate);
  }
  LaunchScope ls(c, KZFWD);
  k_drT<<<(unsigned)(((long long)s.nf * s.S + 255) / 256), 256, 0, c->stream>>>(c->Gdr, Xb, s,
                                                                                  p.rad);
}

}  // namespace tc
