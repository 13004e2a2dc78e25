// Pieces shared by the tensor-core transform kernels (theta_tc.cu,
// zinv_tc.cu): the 7-slice BF16 split of an FP64 operand (Ozaki et al.,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication", Numer. Algorithms 59, 2012), the shared-memory
// operand layout of tcgen05.mma, the bounded mbarrier wait, the issue loop of
// the slice products and the exact recombination of their level sums.
//
// A tile is a product D = A B with A (kTcM rows x kTcK coefficients) a DFT
// matrix with entries in [-1, 1], streamed from global memory as 7 slices of
// kTcChunks chunks each, and B (kTcK coefficients x kTcN data columns) the
// data, sliced in shared memory.  Level L = i + j of the slice products
// a_i b_j lands in TMEM column block L (kTcN columns each, lane = row of A).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

namespace tc {
namespace {

constexpr int kTcM = 128;      // rows of A per MMA (zero rows beyond the transform's length)
constexpr int kTcK = 96;       // real coefficients per data column, padded with zeros
constexpr int kTcN = 32;       // data columns per tile (zero columns beyond those used)
constexpr int kTcS = 7;        // slices of each operand
constexpr int kTcLev = 7;      // level blocks of kTcN TMEM columns each
constexpr int kTcKc = 32;      // coefficients per streamed chunk of a DFT-matrix slice
constexpr int kTcChunks = kTcK / kTcKc;   // 3 per slice
constexpr int kTcStages = kTcChunks * kTcS;   // 21
constexpr int kTcRing = 4;     // chunks in flight (the default ring depth)
// Operand layouts in shared memory (K-major, no swizzle): core matrices of 8
// rows x 16 bytes (8 BF16), the K-neighbour of a core matrix 128 B further,
// the next group of 8 rows one K extent further.
constexpr int kTcBSlice = (kTcN / 8) * (kTcK / 8) * 128;       // 6144 B per data slice
constexpr int kTcBBytes = kTcS * kTcBSlice;                     // 43008
constexpr int kTcAChunk = (kTcM / 8) * (kTcKc / 8) * 128;      // 8192 B per chunk
constexpr int kTcTmemCols = 256;
constexpr long long kTcWaitNs = 1000000000LL;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int b_off(int n, int k) {   // data operand, one slice
  return ((n >> 3) * (kTcK / 8) + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) |
         ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned phase) {
  unsigned ok = 0;
  const unsigned long long t0 = global_ns();
  while (true) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
    if (ok) return true;
    if ((long long)(global_ns() - t0) > kTcWaitNs) return false;
  }
}

// round(|x| 2^(56 - E)) for finite x with |x| < 2^E (ties away from zero).
__device__ __forceinline__ unsigned long long scaled_mag(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  if (be) mant |= 1ull << 52;
  // |x| = mant 2^(ex - 52), ex = max(be, 1) - 1023: result mant 2^(ex + 4 - E)
  const int sh = max(be, 1) - 1023 + 4 - E;
  if (sh >= 0) return mant << sh;            // sh <= 3 since |x| < 2^E
  const int rs = -sh;
  if (rs >= 54) return 0ull;                 // mant + 2^(rs-1) < 2^rs
  return (mant + (1ull << (rs - 1))) >> rs;
}

// The 7 slices of x / 2^E as FP32 bit patterns of integers (slice 0 the most
// significant): q = round(|x| 2^(56 - E)) = sum_j d_j 256^(6 - j) with
// balanced digits d_1..d_6 in [-128, 127] and d_0 in [-128, 256].  Adding
// 0x80 to each of the 7 low bytes of q carries exactly where a digit borrows,
// so the bytes t_b of t = q + 0x0080808080808080 give d = t_b - 128 (the top
// digit t_6 + 256 t_7 - 128).  Each digit is formed in FP32 from the pattern
// 0x4B4000tt = 1.5 2^23 + tt, scaled by the sign of x: exact, and exact in
// BF16 (at most 8 significant bits).
__device__ __forceinline__ void slice_value(double x, int E, unsigned out[kTcS]) {
  const unsigned long long t = scaled_mag(x, E) + 0x0080808080808080ull;
  const unsigned lo = (unsigned)t, hi = (unsigned)(t >> 32);
  const float sg = __uint_as_float(0x3F800000u |
                                   ((unsigned)((unsigned long long)__double_as_longlong(x) >> 32) &
                                    0x80000000u));   // -1 or 1: the sign bit of x
  const float c0 = -12583040.0f * sg;        // -(1.5 2^23 + 128)
#pragma unroll
  for (int b = 0; b < 4; ++b)   // bytes 0..3 -> slices 6..3
    out[kTcS - 1 - b] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B40u, 0x5460 | b)), sg, c0));
#pragma unroll
  for (int b = 0; b < 2; ++b)   // bytes 4, 5 -> slices 2, 1
    out[2 - b] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B40u, 0x5460 | b)), sg, c0));
  out[0] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B40u, 0x5432)), sg, c0));
}

// |x| = mag 2^eu with mag < 2^53 an integer (finite x): the significand and
// the exponent of its last place.
__device__ __forceinline__ unsigned long long mag_of(double x, int &eu) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  if (be) mant |= 1ull << 52;
  eu = max(be, 1) - 1075;
  return mant;
}

// round(mag 2^(eu + 56 - E)) for mag < 2^62 and mag 2^eu < 2^E (ties away
// from zero): the value's 56-bit magnitude in units of 2^(E - 56).
__device__ __forceinline__ unsigned long long scaled_int(unsigned long long mag, int eu, int E) {
  const int sh = eu + 56 - E;
  if (sh >= 0) return mag << sh;             // < 2^56 since mag 2^eu < 2^E
  const int rs = -sh;
  if (rs >= 63) return 0ull;                 // mag + 2^(rs-1) < 2^rs
  return (mag + (1ull << (rs - 1))) >> rs;
}

// The 7 slices of the value with 56-bit magnitude q (units of 2^(E - 56))
// and sign neg, as slice_value forms them.
__device__ __forceinline__ void slice_int(unsigned long long q, bool neg, unsigned out[kTcS]) {
  const unsigned long long t = q + 0x0080808080808080ull;
  const unsigned lo = (unsigned)t, hi = (unsigned)(t >> 32);
  const float sg = neg ? -1.0f : 1.0f;
  const float c0 = -12583040.0f * sg;        // -(1.5 2^23 + 128)
#pragma unroll
  for (int b = 0; b < 4; ++b)   // bytes 0..3 -> slices 6..3
    out[kTcS - 1 - b] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B40u, 0x5460 | b)), sg, c0));
#pragma unroll
  for (int b = 0; b < 2; ++b)   // bytes 4, 5 -> slices 2, 1
    out[2 - b] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B40u, 0x5460 | b)), sg, c0));
  out[0] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B40u, 0x5432)), sg, c0));
}

// Nearest double to a 64-bit integer, as bits (round to nearest even).
__device__ __forceinline__ unsigned long long ll_to_double_bits(long long v) {
  if (v == 0) return 0ull;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(u);
  u <<= lz;                                             // bit 63 set
  unsigned long long frac = (u >> 11) & 0xFFFFFFFFFFFFFull;
  const unsigned long long rb = (u >> 10) & 1ull, st = u & 0x3FFull;
  unsigned long long bits = ((unsigned long long)(63 - lz + 1023) << 52) + frac;
  if (rb && (st || (frac & 1ull))) ++bits;              // carries into the exponent if needed
  return sgn | bits;
}

// Thread 0 of a CTA: the kTcStages chunk stages of A's slices through the
// Ring-deep ring in sA, each followed by its MMAs.  bars[b] (b < Ring) is the
// full barrier of ring buffer b, bars[Ring + b] its free barrier (signalled
// when the products that read it are done), bars[2 Ring] the done barrier.
// load_a(st) starts the copy of chunk st (the first Ring were started by the
// caller).  Stage st = 3 i + ch holds coefficients
// 32 ch .. 32 ch + 31 of slice i; its MMAs take B = data slices 0 .. 6 - i
// (stacked along N) and add into level blocks i .. 6.  consumed counts the
// chunks waited for.  Returns false if a wait ran out; the done barrier is
// signalled either way, once the products issued are done.
template <int Ring, class LoadA>
__device__ __forceinline__ bool issue_slice_products(unsigned long long *bars,
                                                     const unsigned char *sA,
                                                     const unsigned char *sB, unsigned tmem,
                                                     int &consumed, LoadA &&load_a) {
  bool ok = true;
  for (int st = 0; st < kTcStages && ok; ++st) {
    const int i = st / kTcChunks, ch = st - i * kTcChunks, buf = st % Ring;
    if (!tc_wait(smem_u32(&bars[buf]), (unsigned)(st / Ring) & 1u)) {
      ok = false;
      break;
    }
    consumed = st + 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // A = slice i of the DFT matrix (this chunk), B = data slices 0 .. 6 - i
    // stacked along N, D = level blocks i .. 6
    const int nB = (kTcLev - i) * kTcN;
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((unsigned)(nB >> 3) << 17) | ((unsigned)(kTcM >> 4) << 24);
    const unsigned abase = smem_u32(sA + buf * kTcAChunk);
    const unsigned dcol = tmem + (unsigned)(i * kTcN);
#pragma unroll
    for (int t = 0; t < kTcKc / 16; ++t) {
      const unsigned long long ad = tc_desc(abase + t * 256, 128, (kTcKc / 8) * 128);
      const unsigned long long bd =
          tc_desc(smem_u32(sB) + (ch * (kTcKc / 8) + 2 * t) * 128, 128, (kTcK / 8) * 128);
      // the first product (slice 0, coefficients 0..15) initialises every block
      const unsigned en = (st == 0 && t == 0) ? 0u : 1u;
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
          :: "r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&bars[Ring + buf])) : "memory");
    // refill the buffer of the previous stage once its products are done
    if (st >= 1 && st - 1 + Ring < kTcStages) {
      const int pb = (st - 1) % Ring;
      if (!tc_wait(smem_u32(&bars[Ring + pb]), (unsigned)((st - 1) / Ring) & 1u)) {
        ok = false;
        break;
      }
      load_a(st - 1 + Ring);
    }
  }
  // the done barrier is signalled either way, once the products issued are done
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(&bars[2 * Ring])) : "memory");
  return ok;
}

// The seven level blocks of 8 adjacent columns, rows 32 q .. 32 q + 31 (lane
// = row; the calling warp must be warp q of its group of four).
__device__ __forceinline__ void load_levels(unsigned tmem, int q, int col8,
                                            unsigned (&v)[kTcLev][8]) {
#pragma unroll
  for (int L = 0; L < kTcLev; ++L) {
    const unsigned ta = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(L * kTcN + col8 * 8);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[L][0]), "=r"(v[L][1]), "=r"(v[L][2]), "=r"(v[L][3]), "=r"(v[L][4]),
          "=r"(v[L][5]), "=r"(v[L][6]), "=r"(v[L][7])
        : "r"(ta));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Level L holds the integer S_L of weight 2^(-8L): Horner in units of 2^-40,
// the last level rounded to that unit.  Column t of the 8 loaded.
__device__ __forceinline__ long long levels_to_int(const unsigned (&v)[kTcLev][8], int t) {
  long long I = (long long)__float2int_rn(__uint_as_float(v[0][t]));
#pragma unroll
  for (int L = 1; L < kTcLev - 1; ++L)
    I = I * 256 + (long long)__float2int_rn(__uint_as_float(v[L][t]));
  I += (long long)__float2int_rn(__uint_as_float(v[kTcLev - 1][t]) * 0.00390625f);
  return I;
}

// Host: the 7 slices of a kTcM x kTcK matrix y[row kTcK + coefficient] with
// entries in [-1, 1], as BF16 in the A-operand layout, chunk by chunk (slice
// i, coefficients 32 ch .. 32 ch + 31 at (kTcChunks i + ch) kTcAChunk bytes).
// Each entry is rounded to a multiple of 2^-56 and cut into balanced base-256
// digits, the top one in [-256, 256].
inline void pack_dft_slices(const std::vector<long double> &y, std::vector<unsigned short> &out) {
  out.assign((size_t)kTcStages * kTcAChunk / 2, 0);
  auto bf16 = [](int d) -> unsigned short {   // an integer of at most 8 significant bits
    if (d == 0) return 0;
    const unsigned sgn = d < 0 ? 0x8000u : 0u;
    const unsigned a = (unsigned)(d < 0 ? -d : d);
    int e = 0;
    while ((a >> (e + 1)) != 0u) ++e;
    const unsigned mant = e >= 7 ? (a >> (e - 7)) & 0x7Fu : (a << (7 - e)) & 0x7Fu;
    return (unsigned short)(sgn | ((unsigned)(127 + e) << 7) | mant);
  };
  for (int j = 0; j < kTcM; ++j)
    for (int k = 0; k < kTcK; ++k) {
      long long Y = std::llround(std::ldexp(y[(size_t)j * kTcK + k], 56));   // round(y 2^56)
      int dig[kTcS];
      for (int sl = kTcS - 1; sl >= 1; --sl) {
        int lo = (int)(Y & 255ll);
        if (lo >= 128) lo -= 256;
        dig[sl] = lo;
        Y = (Y - lo) / 256;
      }
      dig[0] = (int)Y;
      const int ch = k / kTcKc, kl = k - ch * kTcKc;
      const int off = ((j >> 3) * (kTcKc / 8) + (kl >> 3)) * 128 + (j & 7) * 16 + (kl & 7) * 2;
      for (int sl = 0; sl < kTcS; ++sl)
        out[((size_t)(kTcChunks * sl + ch) * kTcAChunk + off) / 2] = bf16(dig[sl]);
    }
}

}  // namespace
}  // namespace tc
