// Inverse axial transforms of the FP64 nonlinear stage on the tensor cores.
//
// k_zinv (Sec. 2.1: Fourier-Galerkin in z, 3/2-rule padding) forms, for every
// radial level r, field c and azimuthal mode m, the physical values along z
// of three complex columns over the stored axial modes |k| <= K: the
// coefficients a_k, their radial derivative (the 9-point stencil across r)
// and their axial derivative i beta_k a_k,
//   v_l = sum_k a_k e^(2 pi i k l / Nz),   l = 0 .. Nz - 1.
// k_zinv_tc forms these sums as DFT-matrix products on the tensor cores, with
// the 7-slice BF16 split of tc_slices.cuh (exact level sums, exact integer
// combination, one rounding to FP64).
//
// The matrix is folded by the symmetry of the grid.  With
//   P_j = sum_k cos(2 pi k j / Nz) a_k,   Q_j = sum_k sin(2 pi k j / Nz) a_k,
// v_j = P_j + i Q_j and v_(Nz-j) = P_j - i Q_j.  One real matrix, the cosine
// rows j = 0 .. Nz/2 stacked over the sine rows j = 1 .. (Nz-1)/2 (Nz rows in
// all, at most 128), multiplies the real and the imaginary part of each
// complex column as two real data columns of 2K + 1 <= 96 coefficients.  So
// the operand has the shape of the azimuthal kernel's (128 x 96) and streams
// through the same ring, where the unfolded complex product would need twice
// the coefficients.  Each output value is the exact integer sum of one cosine
// and one sine row (both in units of 2^(E-56), E the exponent of the complex
// column), rounded once to FP64.
//
// Data path of one CTA (5 consecutive (r, c, m) columns, m fastest: 30 real
// data columns, 2 of the 32 left zero; numbering the columns across radii
// and fields, rather than tiling each (r, c) plane, makes the tiles fill the
// GPU's CTA slots in nearly whole waves):
//   1. all threads: the value, the d/dr stencil (FP64, the same arithmetic
//      as k_zinv) and i beta a of each coefficient, staged as FP64 over data
//      slices 3..6; then 8 threads per data column slice it into the 7 BF16
//      operand tiles, one exponent per complex column;
//   2. thread 0: the 21 chunks of the matrix's slices through the four-deep
//      ring, 42 MMAs into seven level blocks of TMEM;
//   3. all warps: level sums -> 64-bit integers in shared memory;
//   4. all threads: v_j and v_(Nz-j) from a cosine and a sine row, rounded
//      to FP64, written to V in k_zinv's layout [3 c + d][r][l][m].
// Every wait is bounded (1 s); a wait that runs out sets the timeout flag of
// the context, and the CTA waits (bounded) for its copies in flight, frees
// its tensor memory and returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "fft.cuh"
#include "nl_body.cuh"
#include "tc_internal.h"
#include "tc_slices.cuh"

namespace tc {
namespace {

constexpr int kZtcMB = 5;        // columns per CTA: 5 x 3 complex = 30 real data columns
constexpr int kZtcThreads = 256;
// + 128 bytes to align the operand base: 75904, three CTAs per SM (two of
// them holding tensor memory at a time).  A ring of 8 chunks, two CTAs per
// SM, was slower: 0.161 against 0.131 ms a launch at 64 x 128 x 128 with T.
constexpr int kZtcSmem = kTcBBytes + kTcRing * kTcAChunk + 128;
static_assert(6 * kZtcMB <= kTcN, "data columns of a tile");
static_assert(kTcN * kTcK * 8 <= 4 * kTcBSlice, "FP64 staging fits data slices 3..6");
static_assert(kTcN * kTcM * 8 <= kTcBBytes, "integer level sums fit the data slices");

// I 2^e as the nearest double (I an exact integer): the integer's own
// rounding, then the exponent moved by e; below the normal range a signed
// zero, above it a signed infinity.
__device__ __forceinline__ double scaled_int_to_double(long long I, int e) {
  const unsigned long long b = ll_to_double_bits(I);
  if (!(b & 0x7FFFFFFFFFFFFFFFull)) return 0.0;
  const unsigned long long sg = b & 0x8000000000000000ull;
  const int eb = (int)((b >> 52) & 0x7FF) + e;
  if (eb <= 0) return __longlong_as_double((long long)sg);
  if (eb >= 0x7FF) return __longlong_as_double((long long)(sg | 0x7FF0000000000000ull));
  return __longlong_as_double(
      (long long)((b & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)eb << 52)));
}

__global__ void __launch_bounds__(kZtcThreads, 3)
k_zinv_tc(const double2 *__restrict__ X, double2 *__restrict__ Vout, NLParams p,
          const unsigned char *__restrict__ dft, int *__restrict__ timeout, int arm) {
  const Sizes &s = p.sz;
  // columns g = (r nf + c) NM + m, kZtcMB of them per CTA
  const int g0 = blockIdx.x * kZtcMB;
  const int nm = min(kZtcMB, s.Nr * s.nf * s.NM - g0);
  const int Nz = s.Nz, NK = s.NK;
  const int h = Nz >> 1;          // cosine rows j = 0 .. h
  const int hq = (Nz - 1) >> 1;   // sine rows j = 1 .. hq, at lane h + j
  extern __shared__ __align__(128) unsigned char sm_raw[];
  unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
  unsigned char *sB = sm;
  unsigned char *sA = sm + kTcBBytes;
  __shared__ __align__(8) unsigned long long bars[2 * kTcRing + 1];   // full, free, done
  __shared__ unsigned tmem_s;
  __shared__ int colE[kTcN / 2];
  __shared__ int abort_s;
  __shared__ int colm[kZtcMB], colr[kZtcMB], colc[kZtcMB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < nm) {
    const int g = g0 + tid;
    const int rc = fdiv(g, p.fNM);
    colm[tid] = g - rc * s.NM;
    colr[tid] = rc / s.nf;
    colc[tid] = rc - (rc / s.nf) * s.nf;
  }
  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < 2 * kTcRing + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0's count of chunks whose copies were started / waited for
  int loaded = 0, consumed = 0;
  // chunk st of the matrix's slices into ring buffer st % kTcRing
  auto load_a = [&](int st) {
    if (!arm) return;   // test hook: the chunk copies never start, the waits run out
    loaded = st + 1;
    const int b = st % kTcRing;
    const unsigned bar = smem_u32(&bars[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"((unsigned)kTcAChunk) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(sA + b * kTcAChunk)), "l"(dft + (size_t)st * kTcAChunk),
           "r"((unsigned)kTcAChunk), "r"(bar)
        : "memory");
  };
  if (tid == 0)
    for (int st = 0; st < kTcRing; ++st) load_a(st);

  // 1a. the 30 real data columns in FP64, staged over data slices 3..6:
  // Xs[n kTcK + kk], n = 2 (3 mi + d) + part (part 0 real, 1 imaginary),
  // d = 0 value, 1 d/dr, 2 d/dz; kk the stored axial index
  double *Xs = reinterpret_cast<double *>(sB + 3 * kTcBSlice);
  {
    for (int t = tid; t < nm * NK; t += blockDim.x) {
      const int mi = fdiv(t, p.fNK);
      const int kk = t - mi * NK;
      const int r = colr[mi], c = colc[mi];
      const int st = p.rad.s0[r];
      const double *d1 = p.rad.D1 + r * kStencil;
      const double2 *Xc = X + (long long)c * s.S;
      const long long nX = (long long)(s.nf - c) * s.S;   // entries of X from Xc on
      const long long col = (long long)colm[mi] * NK + kk;
      double2 val = {0.0, 0.0}, dr = {0.0, 0.0};
#pragma unroll
      for (int q = 0; q < kStencil; ++q) {
        const long long ix = (long long)(st + q) * s.nmode + col;
        const double2 x = dbg_in(ix, nX, DBG_ZINV_X) ? Xc[ix] : double2{0.0, 0.0};
        dr.x += d1[q] * x.x;
        dr.y += d1[q] * x.y;
        if (st + q == r) val = x;
      }
      const double beta = p.betak[kk];   // alpha k, as k_zinv forms it
      double *o = Xs + (6 * mi) * kTcK + kk;
      o[0] = val.x;
      o[kTcK] = val.y;
      o[2 * kTcK] = dr.x;
      o[3 * kTcK] = dr.y;
      o[4 * kTcK] = -beta * val.y;
      o[5 * kTcK] = beta * val.x;
    }
  }
  __syncthreads();
  // 1b. slicing.  Thread t: data column n = t / 8, part s8 = t % 8, holding
  // coefficients 32 g + 4 s8 .. + 3 for g = 0..2 (one 8-byte store per slice
  // and group).  The 16 threads of a complex column share its exponent.
  {
    const int n = tid >> 3, s8 = tid & 7;
    const bool colv = n < 6 * nm;
    double xv[12];
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 32 * g + 4 * s8 + e;
        xv[4 * g + e] = (colv && k < NK) ? Xs[n * kTcK + k] : 0.0;
      }
    __syncthreads();   // the staging is read: the slices may overwrite it
    unsigned long long mb = 0ull;
#pragma unroll
    for (int u = 0; u < 12; ++u)
      mb = max(mb, (unsigned long long)__double_as_longlong(xv[u]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int E = mb ? (int)((mb >> 52) & 0x7FF) - 1022 : 0;   // max |x| < 2^E
    if ((tid & 15) == 0) colE[tid >> 4] = E;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      unsigned f[4][kTcS];
#pragma unroll
      for (int v = 0; v < 4; ++v) slice_value(xv[4 * g + v], E, f[v]);
      const int k0 = 32 * g + 4 * s8;
#pragma unroll
      for (int sl = 0; sl < kTcS; ++sl) {
        // BF16 = top half of the FP32 digit; the lower k in the lower half
        uint2 w;
        w.x = __byte_perm(f[0][sl], f[1][sl], 0x7632);
        w.y = __byte_perm(f[2][sl], f[3][sl], 0x7632);
        *reinterpret_cast<uint2 *>(sB + sl * kTcBSlice + b_off(n, k0)) = w;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  // tensor memory only now (another CTA on this SM may hold it meanwhile: the
  // allocation waits for it)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_s)), "r"(kTcTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_s;

  // 2. the slice products (thread 0 issues them)
  if (tid == 0) {
    if (!issue_slice_products<kTcRing>(bars, sA, sB, tmem, consumed, load_a)) abort_s = 1;
  }
  __syncthreads();
  // the same verdict in every thread
  const bool done = __syncthreads_and(tc_wait(smem_u32(&bars[2 * kTcRing]), 0u)) && abort_s == 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done && tid == 0) {
    atomicOr(timeout, 1);
    // wait (bounded) for the copies still in flight, so that none lands
    // after the CTA has left
    for (int st = consumed; st < loaded; ++st)
      if (!tc_wait(smem_u32(&bars[st % kTcRing]), (unsigned)(st / kTcRing) & 1u)) break;
  }
  // 3. level sums -> integers Ib[n][row] in units of 2^(E - 56), over the data
  // slices (the products are done).  Warp w reads TMEM lanes 32 (w % 4) ..;
  // warps 0-3 take columns 0-15, warps 4-7 columns 16-31.
  long long *Ib = reinterpret_cast<long long *>(sm);
  if (done) {
    const int wq = warp & 3;
    const int j = wq * 32 + lane;
#pragma unroll 1
    for (int cc = 0; cc < kTcN / 16; ++cc) {
      const int cb = (warp >> 2) * (kTcN / 16) + cc;
      unsigned v[kTcLev][8];
      load_levels(tmem, wq, cb, v);
#pragma unroll
      for (int t = 0; t < 8; ++t) Ib[(cb * 8 + t) * kTcM + j] = levels_to_int(v, t);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kTcTmemCols) : "memory");
  if (!done) return;

  // 4. v_j = P_j + i Q_j and v_(Nz-j) = P_j - i Q_j from the integer sums of
  // the real (n) and imaginary (n + 1) data columns; one rounding each
  const long long vsz = 3LL * s.nf * s.Nr * Nz * s.NM;
  for (int t = tid; t < (h + 1) * 3 * nm; t += blockDim.x) {
    const int q = t / nm;
    const int mi = t - q * nm;
    const int j = q / 3;
    const int d = q - 3 * j;
    const int n = 2 * (3 * mi + d);
    const long long Pr = Ib[n * kTcM + j], Pi = Ib[(n + 1) * kTcM + j];
    const bool mirror = j >= 1 && j <= hq;
    long long Qr = 0, Qi = 0;
    if (mirror) {
      Qr = Ib[n * kTcM + h + j];
      Qi = Ib[(n + 1) * kTcM + h + j];
    }
    const int e = colE[n >> 1] - 56;
    const long long io =
        (((long long)(3 * colc[mi] + d) * s.Nr + colr[mi]) * Nz + j) * s.NM + colm[mi];
    if (dbg_in(io, vsz, DBG_ZINV_V))
      Vout[io] = double2{scaled_int_to_double(Pr - Qi, e), scaled_int_to_double(Pi + Qr, e)};
    if (mirror) {
      const long long im = io + (long long)(Nz - 2 * j) * s.NM;   // row Nz - j
      if (dbg_in(im, vsz, DBG_ZINV_V))
        Vout[im] = double2{scaled_int_to_double(Pr + Qi, e), scaled_int_to_double(Pi - Qr, e)};
    }
  }
}

}  // namespace

// The folded axial DFT matrix for Nz, K: row j <= Nz/2 holds cos(2 pi k j /
// Nz), row Nz/2 + j (1 <= j <= (Nz-1)/2) holds sin(2 pi k j / Nz), column kk
// the stored axial index (k = kk for kk <= K, kk - (2K+1) above); rows from
// Nz and columns from 2K+1 on are zero.  21 chunks of the A-operand layout.
void build_zinv_dft(int Nz, int K, std::vector<unsigned short> &out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int NK = 2 * K + 1, h = Nz / 2;
  std::vector<long double> y((size_t)kTcM * kTcK, 0.0L);
  for (int row = 0; row < Nz && row < kTcM; ++row)
    for (int kk = 0; kk < NK && kk < kTcK; ++kk) {
      const long long k = kk <= K ? kk : kk - NK;
      const bool sine = row > h;
      const long long j = sine ? row - h : row;
      const long long kj = ((k * j) % Nz + Nz) % Nz;   // exact reduction of the angle
      const long double ang = 2.0L * pi * (long double)kj / Nz;
      y[(size_t)row * kTcK + kk] = sine ? std::sin(ang) : std::cos(ang);
    }
  pack_dft_slices(y, out);
}

bool zinv_tc_supported(const Sizes &s) { return s.Nz <= kTcM && s.NK <= kTcK; }

size_t zinv_tc_table_bytes() { return (size_t)kTcStages * kTcAChunk; }

void setup_zinv_tc() { allow_smem(k_zinv_tc); }

void launch_zinv_tc(cudaStream_t st, const double2 *X, double2 *V, const NLParams &p,
                    const unsigned char *dft, int *timeout, bool arm) {
  const Sizes &s = p.sz;
  const int ncol = s.Nr * s.nf * s.NM;
  k_zinv_tc<<<(ncol + kZtcMB - 1) / kZtcMB, kZtcThreads, kZtcSmem, st>>>(X, V, p, dft, timeout,
                                                                          arm ? 1 : 0);
}

}  // namespace tc
