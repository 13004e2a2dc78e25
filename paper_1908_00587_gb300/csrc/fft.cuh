// Batched complex FFTs of length N = 2^a 3^b 5^c held in shared memory.
//
// Self-sorting (Stockham) mixed-radix passes with radices 8, 4, 2, 3, 5: pass
// p of radix R with stride Ns (product of the earlier radices) takes, for each
// butterfly j < N/R, the R inputs x[j + q N/R], multiplies input q by
// w^(q (j mod Ns)) with w = exp(s 2 pi i / (Ns R)), applies a length-R DFT and
// stores output p at (j div Ns) Ns R + (j mod Ns) + p Ns.  Ping-pong between
// two shared buffers; every thread of the CTA cooperates on the whole batch.
// s = -1 is the forward transform, s = +1 the (unnormalised) inverse.
#pragma once

#include <cuda_runtime.h>

#include "tc_internal.h"

namespace tc {

template <typename T>
struct V2t;
template <>
struct V2t<double> {
  using type = double2;
};
template <>
struct V2t<float> {
  using type = float2;
};

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename V>
__device__ __forceinline__ V csub(V a, V b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// a * (S i), S = +-1
template <int S, typename V>
__device__ __forceinline__ V mul_si(V a) {
  return S > 0 ? V{-a.y, a.x} : V{a.y, -a.x};
}

// Length-R DFTs, out_p = sum_q v_q exp(S 2 pi i p q / R), in place.
template <int S, typename V>
__device__ __forceinline__ void dft2(V *v) {
  V a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int S, typename V>
__device__ __forceinline__ void dft4(V *v) {
  V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  V t2 = cadd(v[1], v[3]), t3 = mul_si<S>(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

// Cosine-tangent form of a twiddle w = c (1 + i t), c = cos, t = tan of its
// angle: w v = c (v + i t v).  Forming v + i t v takes two FMAs and applying c
// while adding into a butterfly output one FMA per component, so a twiddled
// radix-2 step costs 6 FMAs instead of a complex product (4) plus 4 additions
// (Linzer and Feig, "Modified FFTs for fused multiply-add architectures",
// Math. Comp. 60, 1993).  With FMA the result carries the usual complex-product
// error for every angle: c t = sin to rounding, and the rounding of v + i t v
// is scaled back by c.  The tables keep |c| >= 2^-60 so that t stays finite.
template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c) {
  if constexpr (sizeof(T) == 8) return __fma_rn(a, b, c);
  else return __fmaf_rn(a, b, c);
}

// v + i t v
template <typename V, typename T>
__device__ __forceinline__ V ct_u(V v, T t) {
  return V{fmat(-t, v.y, v.x), fmat(t, v.x, v.y)};
}

// a + c u and a - c u
template <typename V, typename T>
__device__ __forceinline__ void ct_pm(V a, T c, V u, V &plus, V &minus) {
  plus = V{fmat(c, u.x, a.x), fmat(c, u.y, a.y)};
  minus = V{fmat(-c, u.x, a.x), fmat(-c, u.y, a.y)};
}

// Twiddled length-4 DFT, out_p = sum_q w^q v_q exp(S 2 pi i p q / 4), in place,
// with w = c1 (1 + i t1) and w^2 = c2 (1 + i t2).  Decimation in time:
// v_0 +- w^2 v_2 and v_1 +- w^2 v_3, then w times the latter: 24 FMAs.
template <int S, typename V, typename T>
__device__ __forceinline__ void dft4_ct(V *v, T c1, T t1, T c2, T t2) {
  V y0, y1, p0, p1;
  ct_pm(v[0], c2, ct_u(v[2], t2), y0, y1);
  ct_pm(v[1], c2, ct_u(v[3], t2), p0, p1);
  ct_pm(y0, c1, ct_u(p0, t1), v[0], v[2]);
  // y1 +- (S i) w p1
  const V u = ct_u(p1, t1);
  const T sc = (T)S * c1;
  v[1] = V{fmat(-sc, u.y, y1.x), fmat(sc, u.x, y1.y)};
  v[3] = V{fmat(sc, u.y, y1.x), fmat(-sc, u.x, y1.y)};
}

// Twiddled length-8 DFT, out_p = sum_q w^q v_q exp(S 2 pi i p q / 8), in place.
// ct[0..4] = w^4, w, w^2, g, g^2 with g = w exp(S i pi / 4), each (c, t).
// Pairs q, q + 4 first (v_q +- w^4 v_(q+4)); the even outputs are then the
// twiddled length-4 DFT of the sums with w, the odd ones that of the
// differences with g: 72 FMAs.
template <int S, typename V, typename T>
__device__ __forceinline__ void dft8_ct(V *v, const V *ct) {
  V P[4], Q[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ct_pm(v[q], (T)ct[0].x, ct_u(v[q + 4], (T)ct[0].y), P[q], Q[q]);
  dft4_ct<S>(P, (T)ct[1].x, (T)ct[1].y, (T)ct[2].x, (T)ct[2].y);
  dft4_ct<S>(Q, (T)ct[3].x, (T)ct[3].y, (T)ct[4].x, (T)ct[4].y);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    v[2 * p] = P[p];
    v[2 * p + 1] = Q[p];
  }
}

// Second half of the length-8 DFT: a_q = v_q + v_(q+4), b_q = v_q - v_(q+4) given.
// The odd outputs are the length-4 DFT of g^q b_q with g = exp(S i pi / 4) =
// h (1 + S i): g^2 = S i is a swap, g is the cosine-tangent form with c = h,
// t = S (v + i t v is two additions).
template <int S, typename V>
__device__ __forceinline__ void dft8_tail(V *a, V *b, V *v) {
  using T = decltype(v[0].x);
  const T h = (T)0.70710678118654752440;  // sqrt(2)/2
  dft4<S>(a);
  {
    const V s2 = mul_si<S>(b[2]), s3 = mul_si<S>(b[3]);
    const V y0 = cadd(b[0], s2), y1 = csub(b[0], s2);
    const V p0 = cadd(b[1], s3), p1 = csub(b[1], s3);
    // v + S i v
    const V u0 = V{p0.x - (T)S * p0.y, p0.y + (T)S * p0.x};
    const V u1 = V{p1.x - (T)S * p1.y, p1.y + (T)S * p1.x};
    ct_pm(y0, h, u0, b[0], b[2]);
    const T sh = (T)S * h;
    b[1] = V{fmat(-sh, u1.y, y1.x), fmat(sh, u1.x, y1.y)};
    b[3] = V{fmat(sh, u1.y, y1.x), fmat(-sh, u1.x, y1.y)};
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    v[2 * p] = a[p];
    v[2 * p + 1] = b[p];
  }
}

template <int S, typename V>
__device__ __forceinline__ void dft8(V *v) {
  V a[4], b[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[q] = cadd(v[q], v[q + 4]);
    b[q] = csub(v[q], v[q + 4]);
  }
  dft8_tail<S>(a, b, v);
}

// Length-8 DFT with v_3 = v_4 = 0 (not read).  This is the first pass of a
// transform whose input vanishes on the middle band [3N/8, 5N/8), which a
// dealiased spectrum packed as (0..B, N-B..N-1) does whenever B < 3N/8.
template <int S, typename V>
__device__ __forceinline__ void dft8_zmid(V *v) {
  V a[4], b[4];
  a[0] = v[0];
  b[0] = v[0];
  a[1] = cadd(v[1], v[5]);
  b[1] = csub(v[1], v[5]);
  a[2] = cadd(v[2], v[6]);
  b[2] = csub(v[2], v[6]);
  a[3] = v[7];
  b[3] = V{-v[7].x, -v[7].y};
  dft8_tail<S>(a, b, v);
}

template <int S, typename V>
__device__ __forceinline__ void dft3(V *v) {
  using T = decltype(v[0].x);
  const T s3 = (T)0.86602540378443864676;  // sqrt(3)/2
  V t = cadd(v[1], v[2]);
  V u = csub(v[1], v[2]);
  V a = V{v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
  V b = mul_si<S>(V{s3 * u.x, s3 * u.y});
  v[0] = cadd(v[0], t);
  v[1] = cadd(a, b);
  v[2] = csub(a, b);
}

template <int S, typename V>
__device__ __forceinline__ void dft5(V *v) {
  using T = decltype(v[0].x);
  const T c1 = (T)0.30901699437494742410;   // cos(2 pi/5) = (sqrt5 - 1)/4
  const T c2 = (T)-0.80901699437494742410;  // cos(4 pi/5) = -(sqrt5 + 1)/4
  const T s1 = (T)0.95105651629515357212;   // sin(2 pi/5)
  const T s2 = (T)0.58778525229247312917;   // sin(4 pi/5)
  V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  V t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  V a1 = V{v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
  V a2 = V{v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
  V b1 = mul_si<S>(V{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y});
  V b2 = mul_si<S>(V{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y});
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

template <int R, int S, typename V>
__device__ __forceinline__ void dftR(V *v) {
  if constexpr (R == 2) dft2<S>(v);
  if constexpr (R == 3) dft3<S>(v);
  if constexpr (R == 4) dft4<S>(v);
  if constexpr (R == 5) dft5<S>(v);
  if constexpr (R == 8) dft8<S>(v);
}

// Shared-memory layout of the transforms: element i of a sequence sits at
// i + i/8 and a sequence of length n occupies padlen(n) slots, so the
// stride-R stores of a Stockham pass spread over the banks instead of
// landing in the same ones.
__host__ __device__ __forceinline__ int spad(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int padlen(int n) { return n + (n >> 3) + 1; }

// True when a spectrum packed as entries 0..B and N-B..N-1 of a length-N
// transform (zeros elsewhere) may use the zero-middle first pass.
__host__ __device__ __forceinline__ bool zmid_ok(const FFTPlan &pl, int B) {
  return pl.npass > 0 && pl.radix[0] == 8 && 8 * B < 3 * pl.n;
}

__device__ __forceinline__ int fdiv(int n, FastDiv f) {
  const unsigned u = (unsigned)n;
  const unsigned t = __umulhi(f.m, u);
  return (int)((t + ((u - t) >> f.s1)) >> f.s2);
}

// One Stockham pass (pass p of plan pl, stride Ns) over `batch` transforms
// stored `bstride` apart.  twp: this pass's twiddles, slot i at i Ns + k, so the
// threads of a warp (consecutive k) read consecutive entries: for radix 4 and
// 8 the cosine-tangent slots named in butterfly(), for radix 2, 3 and 5
// w^(q k) as (cos, sin) in slot q - 1.  The
// index arithmetic divides by the plan's fixed divisors with FastDiv.
// ZMID (radix 8, first pass only): inputs q = 3, 4 are known zeros.
// Butterfly j of one transform, s -> d (both the transform's own storage).
template <int R, int S, bool ZMID, typename V>
__device__ __forceinline__ void butterfly(const V *__restrict__ s, V *__restrict__ d, int j,
                                          int nb, int Ns, FastDiv dns,
                                          const V *__restrict__ twp) {
  const int k = j - fdiv(j, dns) * Ns;
  V v[R];
  const int npad = padlen(nb * R);
#pragma unroll
  for (int q = 0; q < R; ++q)
    if (!ZMID || (q != 3 && q != 4))
      v[q] = dbg_in(spad(j + q * nb), npad, DBG_FFT_SMEM) ? s[spad(j + q * nb)] : V{0, 0};
  if (ZMID) {
    if constexpr (R == 8) dft8_zmid<S>(v);
    const int base = j * R;   // Ns = 1
#pragma unroll
    for (int p = 0; p < R; ++p)
      if (dbg_in(spad(base + p), npad, DBG_FFT_SMEM)) d[spad(base + p)] = v[p];
    return;
  }
  using T = decltype(v[0].x);
  if constexpr (R == 4 || R == 8) {
    // cosine-tangent twiddles: slots w, w^2 (radix 4); w^4, w, w^2, g, g^2
    // (radix 8); the inverse conjugates them, t -> -t
    if (Ns > 1) {
      constexpr int NT = R == 4 ? 2 : 5;
      V ct[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        const V w = twp[i * Ns + k];
        ct[i] = V{w.x, (S < 0) ? w.y : -w.y};
      }
      if constexpr (R == 4) dft4_ct<S>(v, (T)ct[0].x, (T)ct[0].y, (T)ct[1].x, (T)ct[1].y);
      else dft8_ct<S, V, T>(v, ct);
    } else {
      dftR<R, S>(v);
    }
  } else {
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const V w = twp[(q - 1) * Ns + k];
        v[q] = (S < 0) ? cmul(v[q], w) : cmulc(v[q], w);
      }
    }
    dftR<R, S>(v);
  }
  const int base = (j - k) * R + k;
#pragma unroll
  for (int p = 0; p < R; ++p)
    if (dbg_in(spad(base + p * Ns), npad, DBG_FFT_SMEM)) d[spad(base + p * Ns)] = v[p];
}

// Thread index rotated by rot (0 <= rot < blockDim.x): the loops below hand
// butterfly t to thread (t - rot) mod blockDim.x, so that a pass with fewer
// butterflies than threads does not always land on the first warps (the
// warps of one index share a scheduler partition in every CTA of the SM).
__device__ __forceinline__ int rot_tid(int rot) {
  const int t = (int)threadIdx.x + rot;
  return t >= (int)blockDim.x ? t - (int)blockDim.x : t;
}

// rot for the tile (bx, by): one warp further per tile, mod 4 warps
__device__ __forceinline__ int tile_rot(int bx, int by) {
  return (((bx + by) & 3) * 32) % (int)blockDim.x;
}

template <int R, int S, bool ZMID, typename V>
__device__ __forceinline__ void stockham_pass(const V *__restrict__ src, V *__restrict__ dst,
                                              const FFTPlan &pl, int p, int Ns, int batch,
                                              int bstride, const V *__restrict__ twp, int rot) {
  const int nb = pl.n / R;
  const int total = nb * batch;
  const FastDiv dnb = pl.div_nb[p], dns = pl.div_ns[p];
  for (int t = rot_tid(rot); t < total; t += blockDim.x) {
    const int b = fdiv(t, dnb);
    const int j = t - b * nb;
    butterfly<R, S, ZMID>(src + b * bstride, dst + b * bstride, j, nb, Ns, dns, twp);
  }
}

// The same passes for a length known at compile time (powers of two 64..512,
// with the plans make_plan gives them: radix 8 first, then 8s, or two 4s, or
// one 4).  The divisions by nb and Ns become shifts and masks, and the padded
// addresses of a butterfly's inputs and outputs become one base plus constant
// offsets: spad(x + c) = spad(x) + c + c/8 whenever c is a multiple of 8.
template <int R, int S, bool ZMID, int N, int NS, typename V>
__device__ __forceinline__ void stockham_pass_fixed(const V *__restrict__ src, V *__restrict__ dst,
                                                    int batch, int bstride,
                                                    const V *__restrict__ twp, int rot) {
  using T = decltype(src[0].x);
  constexpr int nb = N / R;
  static_assert((nb & (nb - 1)) == 0 && nb % 8 == 0, "power-of-two stride, multiple of 8");
  constexpr int in_step = nb + nb / 8;   // spad distance between inputs q and q + 1
  const int total = nb * batch;
  for (int t = rot_tid(rot); t < total; t += blockDim.x) {
    const int bi = t / nb;
    const int j = t - bi * nb;
    const V *s = src + bi * bstride;
    V *d = dst + bi * bstride;
    const int k = j % NS;
    const int sj = spad(j);
    V v[R];
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (!ZMID || (q != 3 && q != 4))
        v[q] = dbg_in(sj + q * in_step, padlen(N), DBG_FFT_SMEM) ? s[sj + q * in_step] : V{0, 0};
    if constexpr (ZMID) {
      dft8_zmid<S>(v);
    } else if constexpr (NS == 1) {
      dftR<R, S>(v);
    } else {
      constexpr int NT = R == 4 ? 2 : 5;
      V ct[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        const V w = twp[i * NS + k];
        ct[i] = V{w.x, (S < 0) ? w.y : -w.y};
      }
      if constexpr (R == 4) dft4_ct<S>(v, (T)ct[0].x, (T)ct[0].y, (T)ct[1].x, (T)ct[1].y);
      else dft8_ct<S, V, T>(v, ct);
    }
    const int base = (j - k) * R + k;
    if constexpr (NS % 8 == 0) {
      const int sb = spad(base);
#pragma unroll
      for (int p = 0; p < R; ++p)
        if (dbg_in(sb + p * (NS + NS / 8), padlen(N), DBG_FFT_SMEM)) d[sb + p * (NS + NS / 8)] = v[p];
    } else if constexpr (NS == 1) {
      // base = j R and R <= 8: the R outputs share base / 8
      const int sb = base + j * R / 8;
#pragma unroll
      for (int p = 0; p < R; ++p)
        if (dbg_in(sb + p, padlen(N), DBG_FFT_SMEM)) d[sb + p] = v[p];
    } else {
#pragma unroll
      for (int p = 0; p < R; ++p)
        if (dbg_in(spad(base + p * NS), padlen(N), DBG_FFT_SMEM)) d[spad(base + p * NS)] = v[p];
    }
  }
}

template <int S, int N, typename V>
__device__ V *fft_batch_fixed(V *a, V *b, const FFTPlan &pl, int batch, int bstride,
                              const V *__restrict__ tw, bool zmid, int rot) {
  // plans of make_plan: 64 = 8 8, 128 = 8 4 4, 256 = 8 8 4, 512 = 8 8 8
  constexpr int R1 = (N == 128) ? 4 : 8;
  constexpr int R2 = (N == 64) ? 0 : (N == 512 ? 8 : 4);
  if (zmid) stockham_pass_fixed<8, S, true, N, 1>(a, b, batch, bstride, tw, rot);
  else stockham_pass_fixed<8, S, false, N, 1>(a, b, batch, bstride, tw, rot);
  __syncthreads();
  stockham_pass_fixed<R1, S, false, N, 8>(b, a, batch, bstride, tw + pl.tw_off[1], rot);
  __syncthreads();
  if constexpr (R2 == 0) {
    return a;
  } else {
    stockham_pass_fixed<R2, S, false, N, 8 * R1>(a, b, batch, bstride, tw + pl.tw_off[2], rot);
    __syncthreads();
    return b;
  }
}

// Full transform of `batch` sequences held in buffer a (b is scratch of the
// same size); tw: the plan's pass-major twiddle table (fill_plan_twiddles).  Returns the buffer holding the result.  All threads of the CTA
// must call it; it ends with a __syncthreads().  zmid: the caller guarantees
// that every input vanishes on [3N/8, 5N/8) and the plan starts with radix 8
// (see zmid_ok); the first pass then skips those inputs.  Lengths 64..512
// take the compile-time passes above.  rot: thread rotation of the passes
// (rot_tid; 0 <= rot < blockDim.x), which changes only which thread computes
// a butterfly.
template <int S, typename V>
__device__ V *fft_batch(V *a, V *b, const FFTPlan &pl, int batch, int bstride,
                        const V *__restrict__ tw, bool zmid = false, int rot = 0) {
  switch (pl.n) {
    case 64: return fft_batch_fixed<S, 64>(a, b, pl, batch, bstride, tw, zmid, rot);
    case 128: return fft_batch_fixed<S, 128>(a, b, pl, batch, bstride, tw, zmid, rot);
    case 256: return fft_batch_fixed<S, 256>(a, b, pl, batch, bstride, tw, zmid, rot);
    case 512: return fft_batch_fixed<S, 512>(a, b, pl, batch, bstride, tw, zmid, rot);
    default: break;
  }
  int Ns = 1;
  for (int p = 0; p < pl.npass; ++p) {
    const int R = pl.radix[p];
    const V *twp = tw + pl.tw_off[p];
    if (p == 0 && zmid) {
      stockham_pass<8, S, true>(a, b, pl, p, Ns, batch, bstride, twp, rot);
    } else {
      switch (R) {
        case 8: stockham_pass<8, S, false>(a, b, pl, p, Ns, batch, bstride, twp, rot); break;
        case 4: stockham_pass<4, S, false>(a, b, pl, p, Ns, batch, bstride, twp, rot); break;
        case 2: stockham_pass<2, S, false>(a, b, pl, p, Ns, batch, bstride, twp, rot); break;
        case 3: stockham_pass<3, S, false>(a, b, pl, p, Ns, batch, bstride, twp, rot); break;
        default: stockham_pass<5, S, false>(a, b, pl, p, Ns, batch, bstride, twp, rot); break;
      }
    }
    __syncthreads();
    V *t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace tc
