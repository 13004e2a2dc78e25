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

#include <cstdio>

#include "fft.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

__device__ __forceinline__ int kval(int kk, int K, int NK) { return kk <= K ? kk : kk - NK; }

// Position of stored axial index kk in a length-Nz FFT array.
__device__ __forceinline__ int kpos(int kk, int K, int NK, int Nz) {
  return kk <= K ? kk : Nz - NK + kk;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
using V2 = typename V2t<T>::type;

template <typename T>
__device__ __forceinline__ void load_tw(V2<T> *dst, const double2 *src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = V2<T>{(T)src[i].x, (T)src[i].y};
}

// V layout: [3*c + d][r][l][m], d = 0 value, 1 d/dr, 2 d/dz.
template <typename T>
__global__ void k_zinv(const double2 *__restrict__ X, V2<T> *__restrict__ Vout, NLParams p) {
  const Sizes &s = p.sz;
  const int m0 = blockIdx.x * p.MB;
  const int nm = min(p.MB, s.NM - m0);
  const int r = blockIdx.y;
  const int c = blockIdx.z;
  const int Nz = s.Nz;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + 3 * p.MB * Nz;
  V2<T> *tw = B + 3 * p.MB * Nz;
  load_tw<T>(tw, p.twz, Nz);
  for (int i = threadIdx.x; i < 3 * nm * Nz; i += blockDim.x) A[i] = V2<T>{0, 0};
  __syncthreads();
  const int st = p.rad.s0[r];
  const double *d1 = p.rad.D1 + r * kStencil;
  for (int t = threadIdx.x; t < nm * s.NK; t += blockDim.x) {
    const int mi = t / s.NK;
    const int kk = t - mi * s.NK;
    const long long col = (long long)(m0 + mi) * s.NK + kk;
    const double2 *Xc = X + (long long)c * s.S;
    const double2 val = Xc[(long long)r * s.nmode + col];
    double2 dr = {0.0, 0.0};
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
      const double2 x = Xc[(long long)(st + q) * s.nmode + col];
      dr.x += d1[q] * x.x;
      dr.y += d1[q] * x.y;
    }
    const double beta = p.alpha * kval(kk, s.K, s.NK);
    const int pos = kpos(kk, s.K, s.NK, Nz);
    A[(3 * mi + 0) * Nz + pos] = V2<T>{(T)val.x, (T)val.y};
    A[(3 * mi + 1) * Nz + pos] = V2<T>{(T)dr.x, (T)dr.y};
    A[(3 * mi + 2) * Nz + pos] = V2<T>{(T)(-beta * val.y), (T)(beta * val.x)};
  }
  __syncthreads();
  V2<T> *res = fft_batch<+1>(A, B, p.pz, 3 * nm, Nz, tw);
  for (int t = threadIdx.x; t < 3 * nm * Nz; t += blockDim.x) {
    const int mi = t % nm;
    const int rest = t / nm;
    const int l = rest % Nz;
    const int d = rest / Nz;
    Vout[(((long long)(3 * c + d) * s.Nr + r) * Nz + l) * s.NM + m0 + mi] = res[(3 * mi + d) * Nz + l];
  }
}

// mode 0: nonlinear products -> W; mode 1: max |u| and max |T| (initial state scaling)
template <typename T>
__global__ void k_theta(const V2<T> *__restrict__ Vin, V2<T> *__restrict__ W, NLParams p,
                        unsigned long long *__restrict__ rate_bits,
                        unsigned long long *__restrict__ norm_bits, int mode) {
  const Sizes &s = p.sz;
  const int l0 = blockIdx.x * p.LB;
  const int nl = min(p.LB, s.Nz - l0);
  const int r = blockIdx.y;
  const int Nt = s.Nt;
  const int npair = 2 * s.nf;       // complex transforms per z-row
  const int nbuf = p.LB * npair;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + nbuf * Nt;
  V2<T> *tw = B + nbuf * Nt;
  load_tw<T>(tw, p.twt, Nt);
  for (int i = threadIdx.x; i < nl * npair * Nt; i += blockDim.x) A[i] = V2<T>{0, 0};
  __syncthreads();
  // pack: buffer (li, c, 0) = value + i dtheta, (li, c, 1) = d/dr + i d/dz
  for (int t = threadIdx.x; t < nl * s.nf * s.NM; t += blockDim.x) {
    const int m = t % s.NM;
    const int rest = t / s.NM;
    const int c = rest % s.nf;
    const int li = rest / s.nf;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const long long fs = (long long)s.Nr * s.Nz * s.NM;
    V2<T> v = Vin[(3 * c + 0) * fs + off];
    V2<T> dr = Vin[(3 * c + 1) * fs + off];
    V2<T> dz = Vin[(3 * c + 2) * fs + off];
    if (m == 0) {  // real DC of a real field
      v.y = 0;
      dr.y = 0;
      dz.y = 0;
    }
    const T fm = (T)m;
    const V2<T> dt = V2<T>{-fm * v.y, fm * v.x};  // i m v
    V2<T> *b0 = A + (li * npair + 2 * c) * Nt;
    V2<T> *b1 = b0 + Nt;
    // Z_m = a_m + i b_m ; Z_{-m} = conj(a_m) + i conj(b_m)
    b0[m] = V2<T>{v.x - dt.y, v.y + dt.x};
    b1[m] = V2<T>{dr.x - dz.y, dr.y + dz.x};
    if (m > 0) {
      b0[Nt - m] = V2<T>{v.x + dt.y, -v.y + dt.x};
      b1[Nt - m] = V2<T>{dr.x + dz.y, -dr.y + dz.x};
    }
  }
  __syncthreads();
  V2<T> *ph = fft_batch<+1>(A, B, p.pt, nl * npair, Nt, tw);
  V2<T> *out = (ph == A) ? B : A;
  const double rr = p.rad.r[r];
  const T inv_r = (T)p.rad.inv_r[r];
  double rate = 0.0, nu = 0.0, nT = 0.0;
  for (int t = threadIdx.x; t < nl * Nt; t += blockDim.x) {
    const int j = t % Nt;
    const int li = t / Nt;
    const V2<T> *b = ph + li * npair * Nt + j;
    const V2<T> r0 = b[0 * Nt], r1 = b[1 * Nt];   // (ur, ur_t), (ur_r, ur_z)
    const V2<T> t0 = b[2 * Nt], t1 = b[3 * Nt];   // (ut, ut_t), (ut_r, ut_z)
    const V2<T> z0 = b[4 * Nt], z1 = b[5 * Nt];   // (uz, uz_t), (uz_r, uz_z)
    const T ur = r0.x, ut = t0.x, uz = z0.x;
    if (mode == 1) {
      nu = fmax(nu, sqrt((double)ur * ur + (double)ut * ut + (double)uz * uz));
      if (s.nf == 4) nT = fmax(nT, fabs((double)b[6 * Nt].x));
      continue;
    }
    const T ut_r = ut * inv_r;
    const T adv_r = ur * r1.x + ut_r * r0.y + uz * r1.y;
    const T adv_t = ur * t1.x + ut_r * t0.y + uz * t1.y;
    const T adv_z = ur * z1.x + ut_r * z0.y + uz * z1.y;
    const T Nr_ = -(adv_r - ut * ut_r);
    const T Nt_ = -(adv_t + ur * ut_r);
    T Nz_ = -adv_z;
    T NT_ = 0;
    if (s.nf == 4) {
      const V2<T> T0 = b[6 * Nt], T1 = b[7 * Nt];
      Nz_ += (T)p.Gr * T0.x;
      NT_ = -(ur * T1.x + ut_r * T0.y + uz * T1.y);
    }
    V2<T> *o = out + li * 2 * Nt + j;
    o[0] = V2<T>{Nr_, Nt_};
    o[Nt] = V2<T>{Nz_, NT_};
    if (rate_bits) {
      const double a = fmax(fabs((double)ur) / p.rad.dr_min[r],
                            fmax(fabs((double)ut) / (rr * p.dth), fabs((double)uz) / p.dz));
      rate = fmax(rate, a);
    }
  }
  if (mode == 1) {
    for (int o = 16; o > 0; o >>= 1) {
      nu = fmax(nu, __shfl_xor_sync(0xffffffffu, nu, o));
      nT = fmax(nT, __shfl_xor_sync(0xffffffffu, nT, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomic_max_pos(&norm_bits[0], nu);
      atomic_max_pos(&norm_bits[1], nT);
    }
    return;
  }
  if (rate_bits) {
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    if ((threadIdx.x & 31) == 0) atomic_max_pos(rate_bits, rate);
  }
  __syncthreads();
  V2<T> *scratch = (out == A) ? B : A;
  V2<T> *sp = fft_batch<-1>(out, scratch, p.pt, nl * 2, Nt, tw);
  // unpack two real transforms: X_m = (Z_m + conj Z_-m)/2, Y_m = (Z_m - conj Z_-m)/(2i)
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  for (int t = threadIdx.x; t < nl * s.NM; t += blockDim.x) {
    const int m = t % s.NM;
    const int li = t / s.NM;
    const V2<T> *z0 = sp + li * 2 * Nt;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const int mm = (Nt - m) % Nt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const V2<T> a = z0[h * Nt + m];
      const V2<T> b = z0[h * Nt + mm];
      const V2<T> x = V2<T>{(T)0.5 * (a.x + b.x), (T)0.5 * (a.y - b.y)};
      const V2<T> y = V2<T>{(T)0.5 * (a.y + b.y), (T)0.5 * (b.x - a.x)};
      W[(2 * h) * fs + off] = x;
      if (2 * h + 1 < s.nf) W[(2 * h + 1) * fs + off] = y;
    }
  }
}

// W layout [g][r][l][m] -> N [g][r][m][kk]
template <typename T>
__global__ void k_zfwd(const V2<T> *__restrict__ W, double2 *__restrict__ N, NLParams p) {
  const Sizes &s = p.sz;
  const int m0 = blockIdx.x * p.MB;
  const int nm = min(p.MB, s.NM - m0);
  const int r = blockIdx.y;
  const int Nz = s.Nz;
  const int nb = s.nf * nm;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + s.nf * p.MB * Nz;
  V2<T> *tw = B + s.nf * p.MB * Nz;
  load_tw<T>(tw, p.twz, Nz);
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  for (int t = threadIdx.x; t < nb * Nz; t += blockDim.x) {
    const int mi = t % nm;
    const int rest = t / nm;
    const int l = rest % Nz;
    const int g = rest / Nz;
    A[(g * nm + mi) * Nz + l] = W[g * fs + ((long long)r * Nz + l) * s.NM + m0 + mi];
  }
  __syncthreads();
  V2<T> *res = fft_batch<-1>(A, B, p.pz, nb, Nz, tw);
  const double scale = 1.0 / ((double)s.Nt * (double)s.Nz);
  for (int t = threadIdx.x; t < nb * s.NK; t += blockDim.x) {
    const int kk = t % s.NK;
    const int rest = t / s.NK;
    const int mi = rest % nm;
    const int g = rest / nm;
    const V2<T> v = res[(g * nm + mi) * Nz + kpos(kk, s.K, s.NK, Nz)];
    N[(long long)g * s.S + (long long)r * s.nmode + (long long)(m0 + mi) * s.NK + kk] =
        double2{(double)v.x * scale, (double)v.y * scale};
  }
}

}  // namespace

void setup_nonlinear(tc_ctx *c) {
  NLParams &p = c->nl;
  const Sizes &s = c->sz;
  const size_t e = sizeof(double2);
  // z kernels: at most ~48 KB per ping-pong buffer
  int MB = (int)(3072 / (3 * s.Nz));
  if (MB < 1) MB = 1;
  if (MB > 8) MB = 8;
  if (MB > s.NM) MB = s.NM;
  p.MB = MB;
  int LB = (int)(4096 / (2 * s.nf * s.Nt));
  if (LB < 1) LB = 1;
  if (LB > 8) LB = 8;
  p.LB = LB;
  c->smem_zinv = (size_t)(2 * 3 * MB * s.Nz + s.Nz) * e;
  c->smem_theta = (size_t)(2 * LB * 2 * s.nf * s.Nt + s.Nt) * e;
  c->smem_zfwd = (size_t)(2 * s.nf * MB * s.Nz + s.Nz) * e;
  cudaFuncSetAttribute(k_zinv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c->smem_zinv);
  cudaFuncSetAttribute(k_theta<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c->smem_theta);
  cudaFuncSetAttribute(k_zfwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c->smem_zfwd);
}

void launch_nonlinear(tc_ctx *c, const double2 *X, double2 *N, unsigned long long *rate_bits,
                      int mode) {
  const Sizes &s = c->sz;
  const NLParams &p = c->nl;
  const int nmb = (s.NM + p.MB - 1) / p.MB;
  {
    LaunchScope ls(c, KZINV);
    k_zinv<double><<<dim3(nmb, s.Nr, s.nf), 256, c->smem_zinv, c->stream>>>(X, c->V, p);
  }
  const int nlb = (s.Nz + p.LB - 1) / p.LB;
  {
    LaunchScope ls(c, KTHETA);
    k_theta<double><<<dim3(nlb, s.Nr), 256, c->smem_theta, c->stream>>>(
        c->V, c->W, p, rate_bits, c->scal->norm_bits, mode);
  }
  if (mode == 1) return;
  LaunchScope ls(c, KZFWD);
  k_zfwd<double><<<dim3(nmb, s.Nr), 256, c->smem_zfwd, c->stream>>>(c->W, N, p);
}

}  // namespace tc
