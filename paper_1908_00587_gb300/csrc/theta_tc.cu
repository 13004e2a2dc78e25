// Azimuthal transforms of the FP64 nonlinear stage on the tensor cores.
//
// The inverse theta transform of k_theta (Sec. 2.1: Fourier-Galerkin in
// theta) is a dense contraction: for every radial level and z row, the
// physical values of each real field are u(theta_j) = sum_k F_jk x_k with
// x_2m = Re a_m, x_2m+1 = Im a_m (Im a_0 = 0) and F_j0 = 1, F_j1 = 0,
// F_j,2m = 2 cos(m theta_j), F_j,2m+1 = -2 sin(m theta_j).  k_theta_tc forms
// these products with tcgen05.mma in BF16 at FP64 accuracy by splitting both
// operands into 7 slices of 8 significant bits (Ozaki et al., "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012):
//   F/2   = 2^-8 sum_i a_i 2^-8i,   x/2^E = 2^-8 sum_j b_j 2^-8j,
// a_i, b_j integers in [-256, 256] (E: exponent of the data column).  The
// products a_i b_j are exact in BF16 x BF16 -> FP32, and so is the sum of all
// pairs of one level L = i + j over the at most 96 coefficients (at most 7
// pairs x 96 terms, below 2^24).  The slices of the data sit one above the
// other along N, so one MMA with A = a_i and B = (b_0 .. b_(6-i)) adds a_i b_j
// to TMEM column block i + j: seven level blocks, each exact.  Levels above 6
// are below 2^-56 of the result and are not formed (28 of the 49 slice
// products).  The level sums are combined exactly in 64-bit integers and
// rounded once to FP64.  The theta derivative is the same product applied to
// i m a_m.
//
// The rest of the stage is k_theta's: the products u.grad u (with curvature
// terms, buoyancy and the CFL rate) in FP64 on the physical grid, then the
// forward theta FFT in FP64 and the unpacking into W.
//
// Data path of one CTA (2 z rows of one radial level, 32 data columns):
//   1. all threads (8 per column): read V, slice the 32 columns into 7 BF16
//      operand tiles in shared memory (K-major core-matrix layout, no
//      swizzle), one exponent per column;
//   2. thread 0: stream the 21 chunks of the DFT matrix's slices (each 128
//      rows x 32 coefficients, 8 KB, already in the operand layout) with 1-D
//      bulk copies into a four-deep ring and issue 7 x 6 MMAs (M 128,
//      N 32 (7 - i), K 16) into the seven level blocks of 32 TMEM columns;
//   3. all warps: read the accumulators (lane = theta row), combine them and
//      write the physical fields (FP64) to shared memory;
//   4. all threads: products, forward FFT, unpack (as k_theta).
// Every wait is bounded (1 s); a wait that runs out sets the timeout flag of
// the context, and the CTA waits (bounded) for its copies in flight, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "nl_body.cuh"
#include "tc_internal.h"
#include "tc_slices.cuh"

namespace tc {
namespace {

constexpr int kTcLB = 2;       // z rows per CTA
constexpr int kTcThreads = 256;
// + 128 bytes to align the base for the tiled TMA copy: 75904, three CTAs per
// SM.  (A ring of 8 chunks, two CTAs per SM, was slower: 0.360 against 0.291
// ms a launch at 64 x 128 x 128 with temperature.)
constexpr int kTcSmem = kTcBBytes + kTcRing * kTcAChunk + 128;

__global__ void __launch_bounds__(kTcThreads, 3)
k_theta_tc(const __grid_constant__ CUtensorMap tmV, double2 *__restrict__ W, NLParams p,
           const unsigned char *__restrict__ dft, unsigned long long *__restrict__ rate_bits,
           int *__restrict__ timeout, int arm) {
  constexpr int LB = kTcLB;
  const Sizes &s = p.sz;
  const int l0 = blockIdx.x * LB;
  const int nl = min(LB, s.Nz - l0);
  const int r = blockIdx.y;
  const int Nt = s.Nt;
  const int Ntp = padlen(Nt);
  const int M = s.M;
  const int ncol = 4 * s.nf;                      // data columns per z row
  extern __shared__ __align__(128) unsigned char sm_raw[];
  unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
  unsigned char *sB = sm;
  unsigned char *sA = sm + kTcBBytes;
  __shared__ __align__(8) unsigned long long bars[2 * kTcRing + 2];   // full, free, done, V
  __shared__ unsigned tmem_s;
  __shared__ int colE[kTcN];
  __shared__ int abort_s;
  __shared__ unsigned long long cfl_cta[3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < 2 * kTcRing + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 3) cfl_cta[tid] = 0ull;
  __syncthreads();
  // thread 0's count of chunks whose copies were started / waited for
  int loaded = 0, consumed = 0;
  // chunk st of the DFT matrix into ring buffer st % kTcRing
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
  // this tile's block of V: one tiled TMA copy of the box {2 NM doubles, 2 z
  // rows, 1 radius, 3 nf planes} (rows past Nz read as zeros) into the space
  // of data slices 4..6, which the slicing below overwrites only after every
  // thread has read its values
  const double2 *Vs = reinterpret_cast<const double2 *>(sB + 4 * kTcBSlice);
  const unsigned vbar = smem_u32(&bars[2 * kTcRing + 1]);
  if (tid == 0) {
    const unsigned vbytes = (unsigned)(3 * s.nf * 2 * s.NM) * 16u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(vbar), "r"(vbytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(smem_u32(Vs)), "l"(reinterpret_cast<unsigned long long>(&tmV)), "r"(0), "r"(l0),
           "r"(r), "r"(0), "r"(vbar)
        : "memory");
    for (int st = 0; st < kTcRing; ++st) load_a(st);
  }

  // 1. the data columns of this tile, sliced.  Thread t: column n = t / 8,
  // part s8 = t % 8.  Column n = li ncol + 4 c + q: z row li, field c, q = 0
  // value, 1 theta derivative, 2 d/dr, 3 d/dz.  Coefficient k = 2 m + h:
  // h = 0 Re a_m, h = 1 Im a_m (Im a_0 taken as 0, as the real inverse FFT
  // does); the thread holds m = 16 g + 2 s8 + {0, 1}, g = 0..2, so that one
  // group g is four adjacent coefficients (one 8-byte store per slice).
  // Each coefficient is held as sign, integer magnitude and the exponent of
  // its last place.  The theta derivative's coefficients i m a_m =
  // (-m Im a_m, m Re a_m) are formed there exactly (the 53-bit significand
  // times m in 64-bit integers, one rounding at the split): no FP64
  // instruction, which in a warp where one column in four takes the
  // derivative would cost the whole warp's turn on the FP64 unit.
  const long long fs = (long long)s.Nr * s.Nz * s.NM;
  // the V block, waited for by every thread (the same verdict in all)
  if (!__syncthreads_and(tc_wait(vbar, 0u))) {
    if (tid == 0) {
      atomicOr(timeout, 1);
      tc_wait(vbar, 0u);   // the V copy, if still in flight (bounded)
      for (int st = consumed; st < loaded; ++st)
        if (!tc_wait(smem_u32(&bars[st % kTcRing]), (unsigned)(st / kTcRing) & 1u)) break;
    }
    return;
  }
  {
    const int n = tid >> 3, s8 = tid & 7;
    const int li = n / ncol, cq = n - li * ncol, c = cq >> 2, q = cq & 3;
    const bool col = li < nl && cq < ncol;
    const int d = q <= 1 ? 0 : q - 1;
    const int base = ((3 * c + d) * 2 + li) * s.NM;   // in the V block
    double2 a[6];
    int et = INT_MIN;   // largest exponent of a leading bit in the column part
    // the data pair of coefficient u: (Re a, Im a), or (-m Im a, m Re a) for
    // the derivative, as magnitudes mag 2^eu (times m) and signs
    auto pair = [&](const double2 &au, int u, int h, int &e, bool &neg) -> unsigned long long {
      const int m = 16 * (u >> 1) + 2 * s8 + (u & 1);
      const double x = (q == 1) == (h == 0) ? au.y : au.x;
      neg = (__double_as_longlong(x) < 0) != (q == 1 && h == 0);
      return mag_of(x, e) * (q == 1 ? (unsigned long long)m : 1ull);
    };
#pragma unroll
    for (int u = 0; u < 6; ++u) {   // all loads first
      const int m = 16 * (u >> 1) + 2 * s8 + (u & 1);
      double2 v = double2{0.0, 0.0};
      if (col && m <= M && dbg_in(base + m, 6LL * s.nf * s.NM, DBG_THETA_V)) {
        v = Vs[base + m];
        if (m == 0) v.y = 0.0;
      }
      a[u] = v;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int e;
        bool neg;
        const unsigned long long mg = pair(a[u], u, h, e, neg);
        if (mg) et = max(et, e + 63 - __clzll((long long)mg));
      }
    }
    __syncthreads();   // the V block is read: the slices may overwrite it
    // exponent of the column: E with max |x| < 2^E (the 8 threads of a column
    // are 8 adjacent lanes)
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) et = max(et, __shfl_xor_sync(0xffffffffu, et, o));
    const int E = et == INT_MIN ? 0 : et + 1;   // 2^et <= max < 2^(et+1) = 2^E
    if (s8 == 0) colE[n] = E;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      unsigned f[4][kTcS];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int e;
        bool neg;
        const unsigned long long mg = pair(a[2 * g + (v >> 1)], 2 * g + (v >> 1), v & 1, e, neg);
        slice_int(scaled_int(mg, e, E), neg, f[v]);
      }
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
  // tensor memory only now, for the products and the read-back (another CTA
  // on this SM may hold it meanwhile: the allocation waits for it)
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
  // 3. accumulators -> physical fields P[n][j] (FP64), lane = theta row.
  // Warp w reads TMEM lanes 32 (w % 4) ..; warps 0-3 take columns 0-15,
  // warps 4-7 columns 16-31.
  double *P = reinterpret_cast<double *>(sm);   // over the data slices: the products are done
  if (done) {
    const int wq = warp & 3;
    const int j = wq * 32 + lane;
#pragma unroll 1
    for (int cc = 0; cc < kTcN / 16; ++cc) {
      const int cb = (warp >> 2) * (kTcN / 16) + cc;
      unsigned v[kTcLev][8];
      load_levels(tmem, wq, cb, v);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int n = cb * 8 + t;
        const long long I = levels_to_int(v, t);
        // value = I 2^-40 2^-16 2^(E+1): F/2 and x/2^E each carry a 2^-8
        unsigned long long bits = ll_to_double_bits(I);
        if (bits & 0x7FFFFFFFFFFFFFFFull) bits += (unsigned long long)(long long)(colE[n] - 55) << 52;
        P[n * kTcM + j] = __longlong_as_double((long long)bits);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kTcTmemCols) : "memory");
  if (!done) return;

  // 4. products on the physical grid (as k_theta), forward FFT, unpack
  double2 *out = reinterpret_cast<double2 *>(sm + kTcN * kTcM * sizeof(double));
  double2 *scratch = out + 2 * LB * Ntp;
  double2 *tw = scratch + 2 * LB * Ntp;
  load_tw<double>(tw, p.twt, p.twt32, Nt);
  const double inv_r = p.rad.inv_r[r];
  unsigned long long mr = 0ull, mt = 0ull, mz = 0ull;
  const bool centrifugal = p.eps_c != 0.0;
  auto bitsabs = [](double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  };
  for (int t = tid; t < nl * Nt; t += blockDim.x) {
    const int li = t / Nt, j = t - li * Nt;
    const double *f = P + (li * ncol) * kTcM + j;   // field c, q at f[(4c + q) kTcM]
    const double ur = f[0], ur_t = f[kTcM], ur_r = f[2 * kTcM], ur_z = f[3 * kTcM];
    const double ut = f[4 * kTcM], ut_t = f[5 * kTcM], ut_r_ = f[6 * kTcM], ut_z = f[7 * kTcM];
    const double uz = f[8 * kTcM], uz_t = f[9 * kTcM], uz_r = f[10 * kTcM], uz_z = f[11 * kTcM];
    const double ut_r = ut * inv_r;
    const double adv_r = ur * ur_r + ut_r * ur_t + uz * ur_z;
    const double adv_t = ur * ut_r_ + ut_r * ut_t + uz * ut_z;
    const double adv_z = ur * uz_r + ut_r * uz_t + uz * uz_z;
    double Nr_ = -(adv_r - ut * ut_r);
    double Nt_ = -(adv_t + ur * ut_r);
    double Nz_ = -adv_z;
    double NT_ = 0.0;
    if (s.nf == 4) {
      const double T = f[12 * kTcM], T_t = f[13 * kTcM], T_r = f[14 * kTcM], T_z = f[15 * kTcM];
      if (centrifugal) {
        const double rho = 1.0 - p.eps_c * T;
        Nr_ *= rho;
        Nt_ *= rho;
        Nz_ *= rho;
      }
      Nz_ += p.Gr * T;
      NT_ = -(ur * T_r + ut_r * T_t + uz * T_z);
    }
    double2 *o = out + li * 2 * Ntp + spad(j);
    o[0] = double2{Nr_, Nt_};
    o[Ntp] = double2{Nz_, NT_};
    if (rate_bits) {
      mr = max(mr, bitsabs(ur));
      mt = max(mt, bitsabs(ut));
      mz = max(mz, bitsabs(uz));
    }
  }
  if (rate_bits) {
    for (int o = 16; o > 0; o >>= 1) {
      mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
      mt = max(mt, __shfl_xor_sync(0xffffffffu, mt, o));
      mz = max(mz, __shfl_xor_sync(0xffffffffu, mz, o));
    }
    if (lane == 0) {
      atomicMax(&cfl_cta[0], mr);
      atomicMax(&cfl_cta[1], mt);
      atomicMax(&cfl_cta[2], mz);
    }
  }
  __syncthreads();
  if (rate_bits && tid == 0) {
    auto val = [](unsigned long long b) { return __longlong_as_double((long long)b); };
    const double rate = fmax(val(cfl_cta[0]) * p.cfl_inv[2 * r],
                             fmax(val(cfl_cta[1]) * p.cfl_inv[2 * r + 1], val(cfl_cta[2]) * p.inv_dz));
    atomicMax(rate_bits, (unsigned long long)__double_as_longlong(rate));
  }
  double2 *sp = fft_batch<-1>(out, scratch, p.pt, nl * 2, Ntp, tw, false, tile_rot(blockIdx.x, r));
  // unpack two real transforms: X_m = (Z_m + conj Z_-m)/2, Y_m = (Z_m - conj Z_-m)/(2i);
  // the factor 1/2 is left to k_zfwd's final scaling (as in k_theta)
  for (int t = tid; t < nl * s.NM; t += blockDim.x) {
    const int li = t / s.NM, m = t - li * s.NM;
    const double2 *z0 = sp + li * 2 * Ntp;
    const long long off = ((long long)r * s.Nz + l0 + li) * s.NM + m;
    const int mm = m == 0 ? 0 : Nt - m;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double2 a = z0[h * Ntp + spad(m)];
      const double2 b = z0[h * Ntp + spad(mm)];
      const double2 x = double2{a.x + b.x, a.y - b.y};
      const double2 y = double2{a.y + b.y, b.x - a.x};
      if (dbg_in((2 * h) * fs + off, (long long)s.nf * fs, DBG_THETA_W)) W[(2 * h) * fs + off] = x;
      if (2 * h + 1 < s.nf && dbg_in((2 * h + 1) * fs + off, (long long)s.nf * fs, DBG_THETA_W))
        W[(2 * h + 1) * fs + off] = y;
    }
  }
}

}  // namespace

// The DFT matrix F/2 for Ntheta = Nt, M = Mmax, in 21 chunks of the A operand
// layout (slice i, coefficients 32 ch .. 32 ch + 31 at (3 i + ch) * kTcAChunk
// bytes).
void build_theta_dft(int Nt, int Mm, std::vector<unsigned short> &out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> y((size_t)kTcM * kTcK, 0.0L);
  for (int j = 0; j < kTcM && j < Nt; ++j)
    for (int k = 0; k < kTcK; ++k) {
      const int m = k >> 1, h = k & 1;   // column k = 2 m + h
      if (m > Mm) continue;
      long double v;
      if (m == 0) {
        v = h ? 0.0L : 0.5L;
      } else {
        const long double ang = 2.0L * pi * (long double)((long long)m * j % Nt) / Nt;
        v = h ? -std::sin(ang) : std::cos(ang);
      }
      y[(size_t)j * kTcK + k] = v;
    }
  pack_dft_slices(y, out);
}

bool theta_tc_supported(const Sizes &s) {
  return s.Nt <= kTcM && 2 * (s.M + 1) <= kTcK && kTcLB * 4 * s.nf <= kTcN;
}

size_t theta_tc_table_bytes() { return (size_t)kTcStages * kTcAChunk; }

void setup_theta_tc() {
  allow_smem(k_theta_tc);
}

// V as a 4-D FP64 tensor for the tiled TMA copy: {2 NM (Re, Im per m), Nz,
// Nr, 3 nf planes}, box {2 NM, 2, 1, 3 nf} (at most 96 x 2 x 1 x 12 doubles,
// 18 KB: the space of three data slices).  Row strides are multiples of 16
// bytes (16 NM per z row).
bool theta_tc_map(void *map, const double2 *V, const Sizes &s) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode || 2 * s.NM > kTcK || 3 * s.nf * 2 * s.NM * 16 > 3 * kTcBSlice) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)(2 * s.NM), (cuuint64_t)s.Nz, (cuuint64_t)s.Nr,
                              (cuuint64_t)(3 * s.nf)};
  const cuuint64_t strides[3] = {(cuuint64_t)s.NM * 16, (cuuint64_t)s.NM * 16 * s.Nz,
                                 (cuuint64_t)s.NM * 16 * s.Nz * s.Nr};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * s.NM), (cuuint32_t)kTcLB, 1u,
                             (cuuint32_t)(3 * s.nf)};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  return encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                const_cast<double2 *>(V), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_theta_tc(cudaStream_t st, const void *map, double2 *W, const NLParams &p,
                     const unsigned char *dft, unsigned long long *rate_bits, int *timeout,
                     bool arm) {
  const Sizes &s = p.sz;
  k_theta_tc<<<dim3((s.Nz + kTcLB - 1) / kTcLB, s.Nr), kTcThreads, kTcSmem, st>>>(
      *static_cast<const CUtensorMap *>(map), W, p, dft, rate_bits, timeout, arm ? 1 : 0);
}

}  // namespace tc
