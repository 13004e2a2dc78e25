// Device bodies of the nonlinear-stage kernels (Sec. 2.1: dealiased
// pseudospectral products), shared by the per-stage kernels of nonlinear.cu
// and the persistent ensemble kernel of ensemble.cu.  Each body computes one
// CTA's tile; the caller passes the tile's block indices and, for the
// transform kernels, the CTA's dynamic shared memory.  All bodies expect 256
// threads except the per-element ones, which take their element index.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "fft.cuh"
#include "tc_internal.h"

namespace tc {
namespace {


// Position of stored axial index kk in a length-Nz FFT array.
__device__ __forceinline__ int kpos(int kk, int K, int NK, int Nz) {
  return kk <= K ? kk : Nz - NK + kk;
}

// n / d and n % d for a divisor with a precomputed FastDiv.
__device__ __forceinline__ int2 divmod(int n, int d, FastDiv f) {
  const int q = fdiv(n, f);
  return int2{q, n - q * d};
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
using V2 = typename V2t<T>::type;

// Zero the entries of ntr padded length-n spectra (stride ld) that the
// packing leaves unwritten, the dealiasing gap B+1 .. n-B-1, except the part
// [3n/8, 5n/8) that a dealiased first pass (zmid) never reads.
template <typename V>
__device__ __forceinline__ void zero_gap(V *A, int ntr, int ld, int n, int B, bool zmid) {
  const int lo = B + 1, hi = n - B - 1;
  if (hi < lo) return;
  int s0 = hi + 1, s1 = hi + 1;   // skipped part [s0, s1)
  if (zmid) {   // zmid_ok: 8 B < 3 n, so lo <= 3n/8 and 5n/8 <= hi + 1
    s0 = 3 * n / 8;
    s1 = 5 * n / 8;
  }
  const int L1 = s0 - lo, L = L1 + (hi + 1 - s1);
  for (int t = threadIdx.x; t < ntr * L; t += blockDim.x) {
    const int tr = t / L, u = t - tr * L;
    const int i = (u < L1) ? lo + u : s1 + (u - L1);
    A[tr * ld + spad(i)] = V{0, 0};
  }
}

// Twiddle table into shared memory: the FP64 table, or for the FP32 kernels
// its FP32 copy (no conversion on the FP64 unit).
template <typename T>
__device__ __forceinline__ void load_tw(V2<T> *dst, const double2 *src, const float2 *src32, int n) {
  if constexpr (sizeof(T) == 4) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src32[i];
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  }
}

// Mixed precision: u = U + u_b with U = (0, U_theta(r), U_z(r)) and Tbar(r)
// the (0,0) mode of u_theta, u_z, T; u_b (everything else, including the
// (0,0) mode of u_r) goes through the FP32 transforms, which supply
// u_b.grad u_b with its curvature terms.  The products in which U or Tbar
// takes part are diagonal in (m, k) and are formed in FP64 in k_zfwd:
//   N_r = -(a u_r - 2 (U_theta/r) u_theta) + [U_theta^2 / r]_(0,0)
//   N_theta = -(a u_theta + (U_theta/r + U_theta') u_r)
//   N_z = -(a u_z + U_z' u_r) + Gr T          N_T = -(a T + Tbar' u_r)
// with a = i (m U_theta / r + beta U_z) and (u, T) the u_b coefficients, the
// buoyancy Gr T on the full temperature.  In exact arithmetic the sum equals
// the dealiased product: multiplying by a function of r creates no new modes.

// Mean profiles of the (0,0) mode and their radial derivatives, one thread per r.
__device__ __forceinline__ void meanprof_body(const double2 *__restrict__ X,
                                              double *__restrict__ prof,
                                              float *__restrict__ prof32, const Sizes &s,
                                              const Radial &rad, int r) {
  if (r >= s.Nr) return;
  const int st = rad.s0[r];
  double dUt = 0.0, dUz = 0.0, dTb = 0.0;
#pragma unroll
  for (int q = 0; q < kStencil; ++q) {
    const long long o = (long long)(st + q) * s.nmode;
    const double w = rad.D1[r * kStencil + q];
    dUt += w * X[s.S + o].x;
    dUz += w * X[2 * s.S + o].x;
    if (s.nf == 4) dTb += w * X[3 * s.S + o].x;
  }
  const long long o = (long long)r * s.nmode;
  prof[r * 8 + 0] = X[s.S + o].x;
  prof[r * 8 + 1] = X[2 * s.S + o].x;
  prof[r * 8 + 2] = dUt;
  prof[r * 8 + 3] = dUz;
  prof[r * 8 + 4] = dTb;
  prof[r * 8 + 5] = (s.nf == 4) ? X[3 * s.S + o].x : 0.0;
  prof32[2 * r + 0] = (float)X[s.S + o].x;
  prof32[2 * r + 1] = (float)X[2 * s.S + o].x;
}

// Mixed precision: the perturbation part of the state in FP32 for the axial
// kernel (one rounding per coefficient instead of FP64 stencil arithmetic):
// the (0,0) modes of u_theta, u_z and T are the FP64 mean profiles and are
// left out (zero), as everything that involves them is formed in FP64.
__device__ __forceinline__ void tofloat_body(const double2 *__restrict__ X,
                                             float2 *__restrict__ X32, const Sizes &s,
                                             long long i) {
  if (i >= (long long)s.nf * s.S) return;
  const int f = (int)(i / s.S);
  const long long mode = (i - (long long)f * s.S) % s.nmode;
  const double2 x = X[i];
  X32[i] = (f != 0 && mode == 0) ? float2{0.0f, 0.0f} : float2{(float)x.x, (float)x.y};
}

// V layout: [3*c + d][r][l][m], d = 0 value, 1 d/dr, 2 d/dz.  X is the state
// in the transform's precision (FP32: k_tofloat's copy, mean profiles removed).
template <typename T>
__device__ __forceinline__ void zinv_body(const V2<T> *__restrict__ X, V2<T> *__restrict__ Vout,
                                          const NLParams &p, unsigned char *smem_raw, int bx,
                                          int by, int bz) {
  const Sizes &s = p.sz;
  const int m0 = bx * p.MB;
  const int nm = min(p.MB, s.NM - m0);
  const int r = by;
  const int c = bz;
  const int Nz = s.Nz;
  const int Np = padlen(Nz);
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + 3 * p.MB * Np;
  V2<T> *tw = B + 3 * p.MB * Np;
  load_tw<T>(tw, p.twz, p.twz32, Nz);
  zero_gap(A, 3 * nm, Np, Nz, s.K, zmid_ok(p.pz, s.K));
  __syncthreads();
  const int st = p.rad.s0[r];
  T d1[kStencil];
#pragma unroll
  for (int q = 0; q < kStencil; ++q) {
    if constexpr (sizeof(T) == 4) d1[q] = p.d1_32[r * kStencil + q];
    else d1[q] = p.rad.D1[r * kStencil + q];
  }
  const FastDiv fnm = (nm == p.MB) ? p.fMB : p.fMBl;
  for (int t = threadIdx.x; t < nm * s.NK; t += blockDim.x) {
    const int mi = fdiv(t, p.fNK);
    const int kk = t - mi * s.NK;
    const long long col = (long long)(m0 + mi) * s.NK + kk;
    const V2<T> *Xc = X + (long long)c * s.S;
    const long long nX = (long long)(s.nf - c) * s.S;   // entries of X from Xc on
    const long long iv = (long long)r * s.nmode + col;
    const V2<T> val = dbg_in(iv, nX, DBG_ZINV_X) ? Xc[iv] : V2<T>{0, 0};
    V2<T> dr = {0, 0};
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
      const long long ix = (long long)(st + q) * s.nmode + col;
      const V2<T> x = dbg_in(ix, nX, DBG_ZINV_X) ? Xc[ix] : V2<T>{0, 0};
      dr.x += d1[q] * x.x;
      dr.y += d1[q] * x.y;
    }
    T beta;
    if constexpr (sizeof(T) == 4) beta = p.beta32[kk];
    else beta = p.alpha * kval(kk, s.K, s.NK);
    const int pos = kpos(kk, s.K, s.NK, Nz);
    if (dbg_in((3 * mi + 2) * Np + spad(pos), 3 * p.MB * Np, DBG_FFT_SMEM)) {
      A[(3 * mi + 0) * Np + spad(pos)] = val;
      A[(3 * mi + 1) * Np + spad(pos)] = dr;
      A[(3 * mi + 2) * Np + spad(pos)] = V2<T>{-beta * val.y, beta * val.x};
    }
  }
  __syncthreads();
  V2<T> *res = fft_batch<+1>(A, B, p.pz, 3 * nm, Np, tw, zmid_ok(p.pz, s.K), tile_rot(bx, by + bz));
  for (int t = threadIdx.x; t < 3 * nm * Nz; t += blockDim.x) {
    const int2 a = divmod(t, nm, fnm);
    const int mi = a.y;
    const int2 b = divmod(a.x, Nz, p.fNz);
    const int l = b.y;
    const int d = b.x;
    const long long io = (((long long)(3 * c + d) * s.Nr + r) * Nz + l) * s.NM + m0 + mi;
    if (dbg_in(io, 3LL * s.nf * s.Nr * Nz * s.NM, DBG_ZINV_V))
      Vout[io] = res[(3 * mi + d) * Np + spad(l)];
  }
}

// mode 0: nonlinear products -> W; mode 1: max |u| and max |T| (initial state scaling)
template <typename T>
__device__ __forceinline__ void theta_body(const V2<T> *__restrict__ Vin, V2<T> *__restrict__ W,
                                           const NLParams &p,
                                           unsigned long long *__restrict__ rate_bits,
                                           unsigned long long *__restrict__ norm_bits, int mode,
                                           unsigned char *smem_raw, int bx, int by) {
  const Sizes &s = p.sz;
  const int l0 = bx * p.LB;
  const int nl = min(p.LB, s.Nz - l0);
  const int r = by;
  const int Nt = s.Nt;
  const int Ntp = padlen(Nt);
  const int npair = 2 * s.nf;       // complex transforms per z-row
  const int nbuf = p.LB * npair;
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + nbuf * Ntp;
  V2<T> *tw = B + nbuf * Ntp;
  using CflBits = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned>::type;
  __shared__ CflBits cfl_cta[3];   // CTA maxima of |u_r|, |u_theta|, |u_z| (bit patterns)
  load_tw<T>(tw, p.twt, p.twt32, Nt);
  zero_gap(A, nl * npair, Ntp, Nt, s.M, zmid_ok(p.pt, s.M));
  if (threadIdx.x < 3) cfl_cta[threadIdx.x] = 0;
  __syncthreads();
  // pack: buffer (li, c, 0) = value + i dtheta, (li, c, 1) = d/dr + i d/dz
  for (int t = threadIdx.x; t < nl * s.nf * s.NM; t += blockDim.x) {
    const int2 a = divmod(t, s.NM, p.fNM);
    const int m = a.y;
    const int2 b = divmod(a.x, s.nf, p.fnf);
    const int c = b.y;
    const int li = b.x;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const long long fs = (long long)s.Nr * s.Nz * s.NM;
    if (!dbg_in((3 * c + 2) * fs + off, 3LL * s.nf * fs, DBG_THETA_V) ||
        !dbg_in((li * npair + 2 * c + 1) * Ntp + spad(Nt - 1), nbuf * Ntp, DBG_FFT_SMEM))
      continue;
    V2<T> v = Vin[(3 * c + 0) * fs + off];
    V2<T> dr = Vin[(3 * c + 1) * fs + off];
    V2<T> dz = Vin[(3 * c + 2) * fs + off];
    if (m == 0) {  // real DC of a real field
      v.y = 0;
      dr.y = 0;
      dz.y = 0;
    }
    const T fm = (T)m;
    V2<T> *b0 = A + (li * npair + 2 * c) * Ntp;
    V2<T> *b1 = b0 + Ntp;
    // Z_m = a_m + i b_m ; Z_{-m} = conj(a_m) + i conj(b_m).  For the value
    // and its theta derivative b = i m a: Z_m = (1 - m) a, Z_{-m} = (1 + m) conj(a)
    b0[spad(m)] = V2<T>{fmat(-fm, v.x, v.x), fmat(-fm, v.y, v.y)};
    b1[spad(m)] = V2<T>{dr.x - dz.y, dr.y + dz.x};
    if (m > 0) {
      b0[spad(Nt - m)] = V2<T>{fmat(fm, v.x, v.x), fmat(-fm, v.y, -v.y)};
      b1[spad(Nt - m)] = V2<T>{dr.x + dz.y, -dr.y + dz.x};
    }
  }
  __syncthreads();
  V2<T> *ph = fft_batch<+1>(A, B, p.pt, nl * npair, Ntp, tw, zmid_ok(p.pt, s.M), tile_rot(bx, by));
  V2<T> *out = (ph == A) ? B : A;
  T inv_r;
  if constexpr (sizeof(T) == 4) inv_r = p.inv_r32[r];
  else inv_r = p.rad.inv_r[r];
  // CFL: running maxima of |u_r|, |u_theta|, |u_z| in the transforms'
  // precision, kept as bit patterns (non-negative floating-point values order
  // like their bits: integer max, no FP64 issue slot); the divisions by the
  // spacings come once per CTA after the loop (division by a positive
  // constant is monotone, so the max is unchanged).  The FP32 form adds the
  // mean profile in FP32: the CFL step then carries FP32 rounding, like the
  // rest of that form's nonlinear stage.
  CflBits mr = 0, mt = 0, mz = 0;
  double nu = 0.0, nT = 0.0;
  // |v| as its bit pattern: the sign bit cleared with an integer mask
  auto bits = [](T v) -> CflBits {
    if constexpr (sizeof(T) == 8) return (CflBits)__double_as_longlong(v) & 0x7fffffffffffffffull;
    else return (CflBits)__float_as_uint(v) & 0x7fffffffu;
  };
  auto val = [](CflBits b) -> double {
    if constexpr (sizeof(T) == 8) return __longlong_as_double((long long)b);
    else return (double)__uint_as_float(b);
  };
  // full velocity for the CFL bound (mixed: the transforms carry u' only;
  // only the FP32 instantiation runs the mixed form)
  const bool mixed = sizeof(T) == 4 && p.mixed;
  T Ut = (T)0, Uz = (T)0;
  if constexpr (sizeof(T) == 4) {
    if (mixed) {
      Ut = p.prof32[2 * r + 0];
      Uz = p.prof32[2 * r + 1];
    }
  }
  const bool centrifugal = p.eps_c != 0.0;   // FP64 form only
  for (int t = threadIdx.x; t < nl * Nt; t += blockDim.x) {
    const int2 a = divmod(t, Nt, p.fNt);
    const int j = a.y;
    const int li = a.x;
    const V2<T> *b = ph + li * npair * Ntp + spad(j);
    if constexpr (sizeof(T) == 8) {
      if (p.phys_out) {   // keep the physical fields for the adjoint of this stage
        const long long io = ((long long)r * s.Nz + l0 + li) * npair * Nt + j;
        double2 *o = p.phys_out + io;
        if (dbg_in(io + (long long)(npair - 1) * Nt, (long long)s.Nr * s.Nz * npair * Nt,
                   DBG_THETA_PHYS))
          for (int q = 0; q < npair; ++q) o[q * Nt] = b[q * Ntp];
      }
    }
    const V2<T> r0 = b[0 * Ntp], r1 = b[1 * Ntp];   // (ur, ur_t), (ur_r, ur_z)
    const V2<T> t0 = b[2 * Ntp], t1 = b[3 * Ntp];   // (ut, ut_t), (ut_r, ut_z)
    const V2<T> z0 = b[4 * Ntp], z1 = b[5 * Ntp];   // (uz, uz_t), (uz_r, uz_z)
    const T ur = r0.x, ut = t0.x, uz = z0.x;
    if (mode == 1) {
      nu = fmax(nu, sqrt((double)ur * ur + (double)ut * ut + (double)uz * uz));
      if (s.nf == 4) nT = fmax(nT, fabs((double)b[6 * Ntp].x));
      continue;
    }
    const T ut_r = ut * inv_r;
    const T adv_r = ur * r1.x + ut_r * r0.y + uz * r1.y;
    const T adv_t = ur * t1.x + ut_r * t0.y + uz * t1.y;
    const T adv_z = ur * z1.x + ut_r * z0.y + uz * z1.y;
    T Nr_ = -(adv_r - ut * ut_r);
    T Nt_ = -(adv_t + ur * ut_r);
    T Nz_ = -adv_z;
    T NT_ = 0;
    if (s.nf == 4) {
      const V2<T> T0 = b[6 * Ntp], T1 = b[7 * Ntp];
      if constexpr (sizeof(T) == 8) {
        if (centrifugal) {   // centrifugal buoyancy (FP64 form only)
          const T rho = (T)1 - (T)p.eps_c * T0.x;
          Nr_ *= rho;
          Nt_ *= rho;
          Nz_ *= rho;
        }
        Nz_ += (T)p.Gr * T0.x;   // mixed: buoyancy added in FP64 in k_zfwd
      }
      NT_ = -(ur * T1.x + ut_r * T0.y + uz * T1.y);
    }
    V2<T> *o = out + li * 2 * Ntp + spad(j);
    o[0] = V2<T>{Nr_, Nt_};
    o[Ntp] = V2<T>{Nz_, NT_};
    if (rate_bits) {
      mr = max(mr, bits(ur));
      mt = max(mt, bits(mixed ? ut + Ut : ut));
      mz = max(mz, bits(mixed ? uz + Uz : uz));
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
  // CTA maxima of the bit patterns (integer operations only), then one thread
  // scales them by the inverse spacings: the max over points of the
  // per-point rates, since scaling by a positive constant is monotone
  if (rate_bits) {
    for (int o = 16; o > 0; o >>= 1) {
      mr = max(mr, (CflBits)__shfl_xor_sync(0xffffffffu, mr, o));
      mt = max(mt, (CflBits)__shfl_xor_sync(0xffffffffu, mt, o));
      mz = max(mz, (CflBits)__shfl_xor_sync(0xffffffffu, mz, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&cfl_cta[0], mr);
      atomicMax(&cfl_cta[1], mt);
      atomicMax(&cfl_cta[2], mz);
    }
  }
  __syncthreads();
  if (rate_bits && threadIdx.x == 0) {
    const double rate = fmax(val(cfl_cta[0]) * p.cfl_inv[2 * r],
                             fmax(val(cfl_cta[1]) * p.cfl_inv[2 * r + 1], val(cfl_cta[2]) * p.inv_dz));
    atomic_max_pos(rate_bits, rate);
  }
  V2<T> *scratch = (out == A) ? B : A;
  V2<T> *sp = fft_batch<-1>(out, scratch, p.pt, nl * 2, Ntp, tw, false, tile_rot(bx, by));
  // unpack two real transforms: X_m = (Z_m + conj Z_-m)/2, Y_m = (Z_m - conj Z_-m)/(2i);
  // the factor 1/2 is left to k_zfwd's final scaling (exact: a power of two)
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  for (int t = threadIdx.x; t < nl * s.NM; t += blockDim.x) {
    const int2 a = divmod(t, s.NM, p.fNM);
    const int m = a.y;
    const int li = a.x;
    const V2<T> *z0 = sp + li * 2 * Ntp;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const int mm = m == 0 ? 0 : Nt - m;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const V2<T> a = z0[h * Ntp + spad(m)];
      const V2<T> b = z0[h * Ntp + spad(mm)];
      const V2<T> x = V2<T>{a.x + b.x, a.y - b.y};
      const V2<T> y = V2<T>{a.y + b.y, b.x - a.x};
      if (dbg_in((2 * h) * fs + off, (long long)s.nf * fs, DBG_THETA_W)) W[(2 * h) * fs + off] = x;
      if (2 * h + 1 < s.nf && dbg_in((2 * h + 1) * fs + off, (long long)s.nf * fs, DBG_THETA_W))
        W[(2 * h + 1) * fs + off] = y;
    }
  }
}

// W layout [g][r][l][m] -> N [g][r][m][kk]
template <typename T>
__device__ __forceinline__ void zfwd_body(const V2<T> *__restrict__ W, double2 *__restrict__ N,
                                          const NLParams &p, unsigned char *smem_raw, int bx,
                                          int by) {
  const Sizes &s = p.sz;
  const int m0 = bx * p.MBf;
  const int nm = min(p.MBf, s.NM - m0);
  const int r = by;
  const int Nz = s.Nz;
  const int Np = padlen(Nz);
  const int nb = s.nf * nm;
  V2<T> *A = reinterpret_cast<V2<T> *>(smem_raw);
  V2<T> *B = A + s.nf * p.MBf * Np;
  V2<T> *tw = B + s.nf * p.MBf * Np;
  load_tw<T>(tw, p.twz, p.twz32, Nz);
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  const FastDiv fnm = (nm == p.MBf) ? p.fMBf : p.fMBfl;
  for (int t = threadIdx.x; t < nb * Nz; t += blockDim.x) {
    const int2 a = divmod(t, nm, fnm);
    const int mi = a.y;
    const int2 b = divmod(a.x, Nz, p.fNz);
    const int l = b.y;
    const int g = b.x;
    const long long iw = g * fs + ((long long)r * Nz + l) * s.NM + m0 + mi;
    if (dbg_in(iw, (long long)s.nf * fs, DBG_ZFWD_W) &&
        dbg_in((g * nm + mi) * Np + spad(l), (long long)s.nf * p.MBf * Np, DBG_FFT_SMEM))
      A[(g * nm + mi) * Np + spad(l)] = W[iw];
  }
  __syncthreads();
  V2<T> *res = fft_batch<-1>(A, B, p.pz, nb, Np, tw, false, tile_rot(bx, by));
  // 1/(Ntheta Nz), times the 1/2 of k_theta's unpacking of paired transforms
  // (set on the host: a division here would cost every warp FP64 turns)
  const double scale = p.zscale;
  if (!p.mixed) {
    for (int t = threadIdx.x; t < nb * s.NK; t += blockDim.x) {
      const int2 a = divmod(t, s.NK, p.fNK);
      const int kk = a.y;
      const int2 b = divmod(a.x, nm, fnm);
      const int mi = b.y;
      const int g = b.x;
      const V2<T> v = res[(g * nm + mi) * Np + spad(kpos(kk, s.K, s.NK, Nz))];
      const long long in = (long long)g * s.S + (long long)r * s.nmode + (long long)(m0 + mi) * s.NK + kk;
      if (dbg_in(in, (long long)s.nf * s.S, DBG_ZFWD_N))
        N[in] = double2{(double)v.x * scale, (double)v.y * scale};
    }
    return;
  }
  // Mixed precision: the FP32 transform (scaled in FP32: 1/(2 Ntheta Nz),
  // exact for power-of-two sizes) plus the FP64 products with the mean profiles of
  // this radial level,
  //   N_r += -(a u_r - 2 (U_theta/r) u_theta) (+ U_theta^2/r for the mean)
  //   N_theta += -(a u_theta + (U_theta/r + U_theta') u_r)
  //   N_z += -(a u_z + U_z' u_r) + Gr T      N_T += -(a T + Tbar' u_r)
  // with a = i al, al = m U_theta/r + beta U_z from a table built once per
  // CTA (it serves every field of a mode).
  V2<T> *scratch = (res == A) ? B : A;
  double *alt = reinterpret_cast<double *>(scratch);   // [mi][kk], MBf NK <= 2 nf MBf Np
  const double *pr = p.prof + r * 8;
  const double ir = p.rad.inv_r[r];
  const double Utr = pr[0] * ir, Uz = pr[1], dUt = pr[2], dUz = pr[3], dTb = pr[4];
  const double c0 = 2.0 * Utr, c1 = Utr + dUt;
  for (int t = threadIdx.x; t < nm * s.NK; t += blockDim.x) {
    const int2 a = divmod(t, s.NK, p.fNK);
    alt[t] = (double)(m0 + a.x) * Utr + p.alpha * kval(a.y, s.K, s.NK) * Uz;
  }
  __syncthreads();
  const T fscale = (T)scale;
  for (int t = threadIdx.x; t < nb * s.NK; t += blockDim.x) {
    const int2 a = divmod(t, s.NK, p.fNK);
    const int kk = a.y;
    const int2 b = divmod(a.x, nm, fnm);
    const int mi = b.y;
    const int g = b.x;
    const int m = m0 + mi;
    const V2<T> v = res[(g * nm + mi) * Np + spad(kpos(kk, s.K, s.NK, Nz))];
    double2 out = double2{(double)(v.x * fscale), (double)(v.y * fscale)};
    const long long i = (long long)r * s.nmode + (long long)m * s.NK + kk;
    const bool mean = (m == 0 && kk == 0);
    const double al = alt[mi * s.NK + kk];
    const double2 ur = p.Xfull[i];
    const double2 zero = {0.0, 0.0};
    // w: the field a multiplies; c, x: the coefficient and field of the other term
    double2 w, x;
    double c;
    if (g == 0) {
      w = ur;
      x = mean ? zero : p.Xfull[s.S + i];
      c = -c0;
    } else if (g == 1) {
      w = mean ? zero : p.Xfull[s.S + i];
      x = ur;
      c = c1;
    } else if (g == 2) {
      w = mean ? zero : p.Xfull[2 * s.S + i];
      x = ur;
      c = dUz;
    } else {
      w = mean ? zero : p.Xfull[3 * s.S + i];
      x = ur;
      c = dTb;
    }
    // out -= i al w + c x
    out.x = fma(al, w.y, out.x);
    out.y = fma(-al, w.x, out.y);
    out.x = fma(-c, x.x, out.x);
    out.y = fma(-c, x.y, out.y);
    if (g == 0 && mean) out.x += Utr * pr[0];
    if (g == 2 && s.nf == 4) {
      const double2 T2 = p.Xfull[3 * s.S + i];
      out.x = fma(p.Gr, T2.x, out.x);
      out.y = fma(p.Gr, T2.y, out.y);
    }
    if (dbg_in((long long)g * s.S + i, (long long)s.nf * s.S, DBG_ZFWD_N)) N[(long long)g * s.S + i] = out;
  }
}

}  // namespace
}  // namespace tc
