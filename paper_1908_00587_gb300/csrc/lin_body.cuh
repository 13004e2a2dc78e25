// Device bodies of the linear-stage kernels (Sec. 2.2: per-mode radial
// solves; the predictor-corrector of Sec. 2.1), shared by the per-stage
// kernels of linear.cu and the persistent ensemble kernel of ensemble.cu.
// Each body computes one CTA's tile or one element; the caller passes the
// tile's block indices or the element index (and shared memory where the
// body needs it).
#pragma once

#include <cuda_runtime.h>

#include "tc_internal.h"

namespace tc {
namespace {

__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 operator*(double a, double2 b) { return {a * b.x, a * b.y}; }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ double2 mul_i(double2 a) { return {-a.y, a.x}; }      // i a
__device__ __forceinline__ double2 div_2i(double2 a) { return {0.5 * a.y, -0.5 * a.x}; }  // a/(2i)

__device__ __forceinline__ void axpy(double &acc, double l, double x) { acc -= l * x; }
__device__ __forceinline__ void axpy(double2 &acc, double l, double2 x) {
  acc.x -= l * x.x;
  acc.y -= l * x.y;
}
__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ double2 scale(double2 a, double s) { return {a.x * s, a.y * s}; }


// Row j of an operator, entries at columns j-8 .. j+8 (a[0..16]).
// kind 0: Poisson (Neumann D1 rows at the walls), 1: Helmholtz (identity rows).
__device__ __forceinline__ void build_row(const Radial &rad, int Nr, int j, int kind, double q2,
                                          double beta2, double idt, double ck, double *a) {
#pragma unroll
  for (int e = 0; e < kBandW; ++e) a[e] = 0.0;
  const int st = rad.s0[j];
  if (j == 0 || j == Nr - 1) {
    if (kind == 1) {
      a[kBand] = 1.0;
    } else {
#pragma unroll
      for (int t = 0; t < kStencil; ++t) a[st + t - j + kBand] = rad.D1[j * kStencil + t];
    }
    return;
  }
  const double ir = rad.inv_r[j];
#pragma unroll
  for (int t = 0; t < kStencil; ++t) {
    const double l = rad.D2[j * kStencil + t] + rad.D1[j * kStencil + t] * ir;
    a[st + t - j + kBand] = (kind == 1) ? -ck * l : l;
  }
  const double d = q2 * ir * ir + beta2;
  if (kind == 1)
    a[kBand] += idt + ck * d;
  else
    a[kBand] -= d;
}

// In-place band LU (Doolittle, no pivoting) of one operator, rows built on the
// fly.  Operator-major storage: L row j at L[(o*Nrp + j)*8], U row j at
// U[(o*Nrp + j)*9]: the inverse diagonal 1/u_jj first, then the 8
// super-diagonals divided by u_jj (U = D U' with U' unit upper triangular),
// so a backward row is x_j = b_j/u_jj - sum_f U'(j, j+f) x_(j+f): one FMA
// behind the newest x on the sweeps' critical path.
__device__ void band_factor(const Radial &rad, int Nr, int kind, double q2, double beta2,
                            double idt, double ck, double *L, double *U, int Nrp, int o) {
  const long long base = (long long)o * Nrp;
  for (int j = 0; j < Nr; ++j) {
    double a[kBandW];
    build_row(rad, Nr, j, kind, q2, beta2, idt, ck, a);
#pragma unroll
    for (int e = 0; e < kBand; ++e) {
      const int i = j - kBand + e;
      if (i < 0) continue;
      const double *Ui = U + (base + i) * (kBand + 1);
      // l = a_e / u_ii; l U(i, i+f) = a_e U'(i, i+f)
      const double ae = a[e];
      a[e] = ae * Ui[0];
#pragma unroll
      for (int f = 1; f <= kBand; ++f) {
        if (e + f < kBandW) a[e + f] -= ae * Ui[f];
      }
    }
    const double inv = 1.0 / a[kBand];
    double *Lj = L + (base + j) * kBand;
    double *Uj = U + (base + j) * (kBand + 1);
#pragma unroll
    for (int e = 0; e < kBand; ++e) Lj[e] = a[e];
    Uj[0] = inv;
#pragma unroll
    for (int f = 1; f <= kBand; ++f) Uj[f] = a[kBand + f] * inv;
  }
}

// Solve with stored factors by one thread, in place on x[j * xs] (set-up use:
// influence data).  The sweep kernel below does the per-step solves.
template <typename V>
__device__ void band_solve(const double *__restrict__ L, const double *__restrict__ U, int Nrp,
                           int o, int Nr, V *__restrict__ x, long long xs) {
  const long long base = (long long)o * Nrp;
  V w[kBand];
#pragma unroll
  for (int e = 0; e < kBand; ++e) w[e] = V{};
  for (int j = 0; j < Nr; ++j) {
    const double *row = L + (base + j) * kBand;
    V acc = x[j * xs];
#pragma unroll
    for (int e = 0; e < kBand; ++e) axpy(acc, row[e], w[e]);
#pragma unroll
    for (int e = 0; e < kBand - 1; ++e) w[e] = w[e + 1];
    w[kBand - 1] = acc;
    x[j * xs] = acc;
  }
#pragma unroll
  for (int e = 0; e < kBand; ++e) w[e] = V{};
  for (int j = Nr - 1; j >= 0; --j) {
    const double *row = U + (base + j) * (kBand + 1);
    V acc = scale(x[j * xs], row[0]);
#pragma unroll
    for (int f = kBand; f >= 1; --f) axpy(acc, row[f], w[f - 1]);
#pragma unroll
    for (int f = kBand - 1; f > 0; --f) w[f] = w[f - 1];
    w[0] = acc;
    x[j * xs] = acc;
  }
}


__device__ __forceinline__ void factor_helm_body(const LinParams &p, const DevScalars *sc, int t) {
  if (!sc->refactor) return;
  if (t >= p.nopH + p.nopT) return;
  const double idt = 1.0 / sc->dt;
  const int K1 = p.sz.K + 1;
  if (t < p.nopH) {
    const int q = t / K1, ak = t % K1;
    const double beta = p.alpha * ak;
    band_factor(p.rad, p.sz.Nr, 1, (double)q * q, beta * beta, idt, kCN, p.LH, p.UH, p.Nrp, t);
    if (t == 0 && p.flux_ug) {
      // axial-flux constraint: response of the (0,0) u_z operator to a unit
      // uniform forcing, zero at the walls
      for (int j = 0; j < p.sz.Nr; ++j) p.flux_ug[j] = (j == 0 || j == p.sz.Nr - 1) ? 0.0 : 1.0;
      band_solve(p.LH, p.UH, p.Nrp, 0, p.sz.Nr, p.flux_ug, 1);
    }
  } else {
    const int o = t - p.nopH;
    const int m = o / K1, ak = o % K1;
    const double beta = p.alpha * ak;
    band_factor(p.rad, p.sz.Nr, 1, (double)m * m, beta * beta, idt, kCN * p.kappaT, p.LT, p.UT,
                p.Nrp, o);
  }
}

// Homogeneous solutions and the inverse influence matrix, per (m, |k|).
__device__ __forceinline__ void influence_body(const LinParams &p, const DevScalars *sc, int o) {
  if (!sc->refactor) return;
  if (o >= p.nopP || o == 0) return;
  const int Nr = p.sz.Nr, K1 = p.sz.K + 1, nop = p.nopP;
  const int m = o / K1, ak = o % K1;
  const Radial &rad = p.rad;
  const long long fs = (long long)Nr * nop;
  double *F = p.infl;   // [8][Nr][nop]
  auto at = [&](int f, int j) -> double & { return F[f * fs + (long long)j * nop + o]; };
  const int oHp = (m + 1) * K1 + ak, oHm = (m >= 1 ? m - 1 : 1) * K1 + ak, oHz = m * K1 + ak;
  for (int s = 0; s < 2; ++s) {
    for (int j = 0; j < Nr; ++j) at(s, j) = (j == (s == 0 ? 0 : Nr - 1)) ? 1.0 : 0.0;
    band_solve<double>(p.LP, p.UP, p.Nrp, o, Nr, &at(s, 0), nop);
    for (int j = 0; j < Nr; ++j) {
      double up = 0.0, um = 0.0, z = 0.0;
      if (j > 0 && j < Nr - 1) {
        const int st = rad.s0[j];
        double d1p = 0.0;
#pragma unroll
        for (int t = 0; t < kStencil; ++t) d1p += rad.D1[j * kStencil + t] * at(s, st + t);
        const double mp = m * at(s, j) * rad.inv_r[j];
        up = -(d1p - mp);
        um = -(d1p + mp);
        z = at(s, j);
      }
      at(2 + 2 * s, j) = up;
      at(3 + 2 * s, j) = um;
      at(6 + s, j) = z;
    }
    band_solve<double>(p.LH, p.UH, p.Nrp, oHp, Nr, &at(2 + 2 * s, 0), nop);
    band_solve<double>(p.LH, p.UH, p.Nrp, oHm, Nr, &at(3 + 2 * s, 0), nop);
    band_solve<double>(p.LH, p.UH, p.Nrp, oHz, Nr, &at(6 + s, 0), nop);
  }
  // A[w][s] = div of homogeneous solution s at wall w (only u_r is non-zero
  // next to the wall; the wall values themselves are zero)
  double A[2][2];
  for (int w = 0; w < 2; ++w) {
    const int j = (w == 0) ? 0 : Nr - 1;
    const int st = rad.s0[j];
    for (int s = 0; s < 2; ++s) {
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < kStencil; ++t) {
        const double ur = 0.5 * (at(2 + 2 * s, st + t) + at(3 + 2 * s, st + t));
        acc += rad.D1[j * kStencil + t] * (rad.r[st + t] * ur);
      }
      A[w][s] = acc * rad.inv_r[j];
    }
  }
  const double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
  const double id = 1.0 / det;
  p.Ainv[0 * nop + o] = A[1][1] * id;
  p.Ainv[1 * nop + o] = -A[0][1] * id;
  p.Ainv[2 * nop + o] = -A[1][0] * id;
  p.Ainv[3 * nop + o] = A[0][0] * id;
}

__device__ __forceinline__ void dt_policy_body(DevScalars *sc, double dt_fixed, double cfl,
                                               double dt_max, double *dt_hist, int hist_cap) {
  const double rate = __longlong_as_double((long long)sc->rate_bits);
  sc->dt_old = sc->dt;
  sc->idt_old = sc->idt;
  sc->rate_last = rate;
  sc->rate_bits = 0ull;
  sc->corr_bits = 0ull;
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else {
    const double dt_star = (rate <= 0.0) ? dt_max : fmin(dt_max, cfl / rate);
    const double prev = sc->dt_prev;
    dt = (prev <= 0.0 || dt_star < prev || dt_star > 1.1 * prev) ? dt_star : prev;
  }
  sc->dt = dt;
  sc->idt = 1.0 / dt;
  sc->dt_prev = dt;
  sc->refactor = (dt != sc->dt_factored) ? 1 : 0;
  if (sc->refactor) sc->dt_factored = dt;
  if (dt_hist && sc->hist_pos < hist_cap) dt_hist[sc->hist_pos++] = dt;
}

// Explicit right-hand side R = Y' + c N of component comp at flat index i.
__device__ __forceinline__ double2 rhs_pm(const double2 *Yb, const double2 *N, long long S,
                                          long long i, int comp) {
  const double2 y = Yb[comp * S + i];
  if (comp == 0) {
    const double2 nr = N[i], nt = N[S + i];
    return y + kCN * double2{nr.x - nt.y, nr.y + nt.x};
  }
  if (comp == 1) {
    const double2 nr = N[i], nt = N[S + i];
    return y + kCN * double2{nr.x + nt.y, nr.y - nt.x};
  }
  return y + kCN * N[comp * S + i];
}

// Y' = X/dt + (1-c) L X + (1-c) N, in +- form, at every node.
//
// L X from the previous stage: at interior nodes of modes other than (0,0)
// the last corrector solved (1/dt' - c kappa L) X = R - G(p) for the current
// X (R = Y'_prev + c N1 its right-hand side, G the pressure gradient of the
// total pressure p, dt' that stage's step), so (1 - c) kappa L X =
// ((1 - c)/c) (X/dt' - R + G).  When that stage is known to have produced
// the current state (sc->rhs_ident), those nodes use it: one D1 stencil on p
// instead of the Laplacian stencil on every field.  The wall rows (Dirichlet
// rows of the stage), the (0,0) mode (solved without pressure, with the wall
// values and, with the flux constraint, an extra forcing) and every other
// case take the stencil.
__device__ __forceinline__ void rhs_body(const double2 *__restrict__ X,
                                         const double2 *__restrict__ N,
                                         double2 *__restrict__ Yb,
                                         const double2 *__restrict__ N1,
                                         const double2 *__restrict__ P, const LinParams &p,
                                         const DevScalars *sc, long long i) {
  const Sizes &s = p.sz;
  if (i >= s.S) return;
  const int j = (int)i / s.nmode;
  const int mode = (int)(i - (long long)j * s.nmode);
  const int m = mode / s.NK, kk = mode % s.NK;
  const double beta = p.betak[kk];
  const double idt = sc->idt;
  const double ir = p.rad.inv_r[j];
  const int st = p.rad.s0[j];
  const double om = 1.0 - kCN;
  const long long S = s.S;
  if (sc->rhs_ident && mode != 0 && j > 0 && j < s.Nr - 1) {
    const double q = om / kCN;
    const double idt_old = sc->idt_old;
    const double *d1 = p.rad.D1 + j * kStencil;
    double2 d1p = {0.0, 0.0};
#pragma unroll
    for (int t = 0; t < kStencil; ++t)
      if (dbg_in((long long)(st + t) * s.nmode + mode, S, DBG_RHS))
        d1p = d1p + d1[t] * P[(long long)(st + t) * s.nmode + mode];
    const double2 pj = P[i];
    const double2 mp = (p.mval[m] * ir) * pj;
    const double2 xr = X[i], xt = X[S + i];
    const double2 xp = {xr.x - xt.y, xr.y + xt.x}, xm = {xr.x + xt.y, xr.y - xt.x};
    const double2 nr = N[i], nt = N[S + i];
    const double2 np = {nr.x - nt.y, nr.y + nt.x}, nm = {nr.x + nt.y, nr.y - nt.x};
    const double2 rp = rhs_pm(Yb, N1, S, i, 0), rm = rhs_pm(Yb, N1, S, i, 1);
    Yb[i] = idt * xp + q * (idt_old * xp - rp + (d1p - mp)) + om * np;
    Yb[S + i] = idt * xm + q * (idt_old * xm - rm + (d1p + mp)) + om * nm;
    {
      const double2 x = X[2 * S + i];
      const double2 rz = rhs_pm(Yb, N1, S, i, 2);
      Yb[2 * S + i] = idt * x + q * (idt_old * x - rz + beta * mul_i(pj)) + om * N[2 * S + i];
    }
    if (s.nf == 4) {
      const double2 x = X[3 * S + i];
      const double2 rT = rhs_pm(Yb, N1, S, i, 3);
      Yb[3 * S + i] = idt * x + q * (idt_old * x - rT) + om * N[3 * S + i];
    }
    return;
  }
  const double *lw = p.rad.Lw + j * kStencil;   // D2 + D1/r of row j
  const double b2 = beta * beta, ir2 = ir * ir;
  // L is real, so L(X+-) = L(X_r) +- i L(X_theta): one stencil per primitive field
  double2 Sx[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll
  for (int t = 0; t < kStencil; ++t) {
    const long long o = (long long)(st + t) * s.nmode + mode;
    if (!dbg_in(o, S, DBG_RHS)) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < s.nf) Sx[c] = Sx[c] + lw[t] * X[c * S + o];
  }
  {
    const double2 xr = X[i], xt = X[S + i];
    const double2 xp = {xr.x - xt.y, xr.y + xt.x}, xm = {xr.x + xt.y, xr.y - xt.x};
    const double2 Sp = {Sx[0].x - Sx[1].y, Sx[0].y + Sx[1].x};   // S_r + i S_theta
    const double2 Sm = {Sx[0].x + Sx[1].y, Sx[0].y - Sx[1].x};   // S_r - i S_theta
    const double2 nr = N[i], nt = N[S + i];
    const double2 np = {nr.x - nt.y, nr.y + nt.x}, nm = {nr.x + nt.y, nr.y - nt.x};
    const double qp = (double)(m + 1) * (m + 1), qm = (double)(m - 1) * (m - 1);
    const double2 Lp = Sp - (qp * ir2 + b2) * xp;
    const double2 Lm = Sm - (qm * ir2 + b2) * xm;
    Yb[i] = idt * xp + om * Lp + om * np;
    Yb[S + i] = idt * xm + om * Lm + om * nm;
  }
#pragma unroll
  for (int c = 2; c < 4; ++c) {
    if (c >= s.nf) break;
    const double2 x = X[c * S + i];
    const double kap = (c == 3) ? p.kappaT : 1.0;
    const double2 L = kap * (Sx[c] - ((double)m * m * ir2 + b2) * x);
    Yb[c * S + i] = idt * x + om * L + om * N[c * S + i];
  }
}


// The radial solves work on split real / imaginary planes (the operators are
// real): plane q of a field holds part q (0 re, 1 im) as [r][mode] doubles,
// so one thread owns one real system and its loads coalesce across modes.

// Poisson right-hand side: div R inside, 0 on the Neumann rows and for (0,0).
// A CTA takes kPrW consecutive modes x kPrL consecutive rows.  The radial
// component R_r = (R+ + R-)/2 that the divergence stencil reads is formed once
// per node of the window [j0 - 8, j0 + kPrL + 8) into shared memory (every
// stencil of the tile lies inside: it starts at clamp(j - 4, 0, Nr - 9), which
// is within 8 rows below j), instead of once per tap.
// With temperature the same kernel writes the T Helmholtz right-hand side
// (it needs no pressure), so the T solve can run with the pressure solve.
constexpr int kPrW = 32, kPrL = 32, kPrThreads = 256;
constexpr int kPrWin = kPrL + 16;   // rows of the R_r window of a k_prhs tile
// Rr: the tile's window, kPrWin * kPrW double2 of shared memory.
__device__ __forceinline__ void prhs_body(const double2 *__restrict__ Yb,
                                          const double2 *__restrict__ N,
                                          double *__restrict__ Ps, double *__restrict__ UT,
                                          const LinParams &p, double2 *Rr, int bx, int by) {
  const Sizes &s = p.sz;
  constexpr int kWin = kPrWin;
  const int tx = threadIdx.x % kPrW, ty = threadIdx.x / kPrW;
  constexpr int kRowsT = kPrThreads / kPrW;
  const int mode = bx * kPrW + tx;
  const int j0 = by * kPrL;
  const long long S = s.S;
  for (int q = ty; q < kWin; q += kRowsT) {
    const int jw = j0 - 8 + q;
    double2 rr = {0.0, 0.0};
    if (mode < s.nmode && jw >= 0 && jw < s.Nr) {
      const long long ii = (long long)jw * s.nmode + mode;
      // R_r = (R+ + R-)/2 = (Y+ + Y-)/2 + c N_r
      const double2 yp = Yb[ii], ym = Yb[S + ii], nr = N[ii];
      rr = double2{0.5 * (yp.x + ym.x) + kCN * nr.x, 0.5 * (yp.y + ym.y) + kCN * nr.y};
    }
    Rr[q * kPrW + tx] = rr;
  }
  __syncthreads();
  if (mode >= s.nmode) return;
  for (int r = ty; r < kPrL; r += kRowsT) {
    const int j = j0 + r;
    if (j >= s.Nr) break;
    const long long i = (long long)j * s.nmode + mode;
    double2 b = {0.0, 0.0};
    if (mode != 0 && j > 0 && j < s.Nr - 1) {
      const int m = mode / s.NK, kk = mode % s.NK;
      const double beta = p.betak[kk];
      const int q0 = p.rad.s0[j] - (j0 - 8);
      const double *dw = p.rad.Dw + j * kStencil;   // (1/r_j) D1 r_s
      double2 acc = {0.0, 0.0};
#pragma unroll
      for (int t = 0; t < kStencil; ++t)
        if (dbg_in((q0 + t) * kPrW + tx, kWin * kPrW, DBG_PRHS))
          acc = acc + dw[t] * Rr[(q0 + t) * kPrW + tx];
      const double2 rt = div_2i(rhs_pm(Yb, N, S, i, 0) - rhs_pm(Yb, N, S, i, 1));
      const double2 rz = rhs_pm(Yb, N, S, i, 2);
      const double ir = p.rad.inv_r[j];
      b = acc + (p.mval[m] * ir) * mul_i(rt) + beta * mul_i(rz);
    }
    if (!dbg_in(i, S, DBG_PRHS)) continue;
    Ps[i] = b.x;
    Ps[S + i] = b.y;
    if (UT) {   // T: Dirichlet rows (wall temperatures in the (0,0) mode)
      double2 bt = {0.0, 0.0};
      if (j == 0 || j == s.Nr - 1) {
        if (mode == 0) bt.x = (j == 0) ? 0.5 : -0.5;
      } else {
        bt = rhs_pm(Yb, N, S, i, 3);
      }
      UT[i] = bt.x;
      UT[S + i] = bt.y;
    }
  }
}

// Helmholtz right-hand sides of u+, u-, u_z, wall values on the wall rows (the
// T right-hand side comes from k_prhs).
// Mode (0,0): slot 0 carries u_theta's equation (u_r = 0), slot 1 is unused.
__device__ __forceinline__ void hrhs_body(const double2 *__restrict__ Yb,
                                          const double2 *__restrict__ N,
                                          const double *__restrict__ Ps, double *__restrict__ U,
                                          const LinParams &p, long long i) {
  const Sizes &s = p.sz;
  if (i >= s.S) return;
  const int j = (int)i / s.nmode;
  const int mode = (int)(i - (long long)j * s.nmode);
  const long long S = s.S;
  const bool wall = (j == 0 || j == s.Nr - 1);
  double2 b[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  if (mode == 0) {
    const bool lo = (j == 0);
    if (wall) {
      b[0] = {lo ? p.Re_i : p.Re_o, 0.0};
      b[2] = {0.0, 0.0};
    } else {
      b[0] = div_2i(rhs_pm(Yb, N, S, i, 0) - rhs_pm(Yb, N, S, i, 1));
      b[2] = rhs_pm(Yb, N, S, i, 2);
    }
    b[1] = {0.0, 0.0};
  } else if (wall) {
    b[0] = b[1] = b[2] = double2{0.0, 0.0};
  } else {
    const int m = mode / s.NK, kk = mode % s.NK;
    const double beta = p.betak[kk];
    const int st = p.rad.s0[j];
    double2 d1p = {0.0, 0.0};
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
      const long long o = (long long)(st + q) * s.nmode + mode;
      if (dbg_in(o, S, DBG_HRHS))
        d1p = d1p + p.rad.D1[j * kStencil + q] * double2{Ps[o], Ps[S + o]};
    }
    const double2 pj = {Ps[i], Ps[S + i]};
    const double2 mp = (p.mval[m] * p.rad.inv_r[j]) * pj;
    b[0] = rhs_pm(Yb, N, S, i, 0) - (d1p - mp);
    b[1] = rhs_pm(Yb, N, S, i, 1) - (d1p + mp);
    b[2] = rhs_pm(Yb, N, S, i, 2) - beta * mul_i(pj);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    U[(2 * c) * S + i] = b[c].x;
    U[(2 * c + 1) * S + i] = b[c].y;
  }
}

// ---------------------------------------------------------------------------
// Batched band sweeps with the factors streamed through shared memory.
//
// One CTA owns kSweepOps consecutive |k| values of one m and one field; its
// 4 kSweepOps threads are the real systems (+k, -k) x (re, im) that share those
// operators.  Thread 0 streams chunks of kSweepRows factor rows of all the
// CTA's operators into a kSweepStages-deep ring with 1-D bulk async copies
// (cp.async.bulk, TMA) that complete on an mbarrier per stage; every thread
// sweeps its system from shared memory while the next chunks are in flight.
// Right-hand sides / solutions stay in the split planes (one load per row,
// prefetched a chunk ahead).  Waits are bounded: past kWaitNs the CTA raises
// DevScalars::timeout, drains its own copies (bounded again) and returns.

constexpr long long kWaitNs = 1000000000LL;   // 1 s
// One operator's chunk in the ring: kSweepRows rows of up to kBand + 1
// doubles plus 2 doubles of padding, so the 8 operators a warp reads sit in
// distinct shared-memory banks (unpadded, their blocks are a multiple of
// 128 bytes apart and every row load is an 8-way bank conflict).  The pad
// keeps each block 16-byte aligned for the bulk copies.
constexpr int kSweepOpDoubles = kSweepRows * (kBand + 1) + 2;
constexpr int kSweepStageDoubles = kSweepOps * kSweepOpDoubles;
constexpr size_t kSweepSmem = sizeof(double) * kSweepStages * kSweepStageDoubles;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase `phase` of a barrier to complete.
__device__ bool mbar_wait(unsigned bar, unsigned phase) {
  if (mbar_test(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    __nanosleep(64);
    if (mbar_test(bar, phase)) return true;
    if ((long long)(global_ns() - t0) > kWaitNs) return false;
  }
}

struct SweepField {
  const double *L, *U;   // factors of this field's operators
  double *x;             // re plane; the im plane follows at x + S
  int qshift;            // operator row q = m + qshift (|.|, 0 -> 1 when m = 0 for u-)
  int skip00;            // 1: mode (0,0) has no system (pressure)
  int nop;               // operators stored in L and U (index checks of the debug build)
};

struct SweepArgs {
  SweepField f[4];
  int Nr, Nrp, K, NK, nmode;
  long long S;
  int arm;               // 0 only in the timeout self-test: never start the copies
};

template <int W>   // 8: L blocks (forward), 9: U blocks (backward)
__device__ __forceinline__ void arm_chunk(unsigned bar, double *dst, const double *src, int Nrp,
                                          int o0, int nops, int j0, int nop_total) {
  const unsigned bytes = (unsigned)(kSweepRows * W * sizeof(double));
  // debug build: a chunk past the stored operators is not copied and the
  // barrier expects only the copies made (the wait still completes)
  int ncopy = nops;
  if (!dbg_in((long long)(o0 + nops - 1) * Nrp + j0 + kSweepRows - 1, (long long)nop_total * Nrp,
              DBG_SWEEP_COPY))
    ncopy = 0;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(bar), "r"(bytes * (unsigned)ncopy) : "memory");
  for (int g = 0; g < ncopy; ++g) {
    const double *s = src + ((long long)(o0 + g) * Nrp + j0) * W;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(dst + g * kSweepOpDoubles)), "l"(s), "r"(bytes), "r"(bar) : "memory");
  }
}

// Envelope of the factors.  Row j of every radial operator is a 9-point
// stencil starting at column clamp(j - 4, 0, Nr - 9) (or a boundary row of the
// same reach), so rows j < Nr - 4 reach at most 4 columns below the diagonal
// and columns c > 8 at most 4 rows above it.  LU without pivoting keeps that
// envelope: L rows j < Nr - 4 and U rows j >= 4 hold exact zeros in their 4
// outermost entries.  The sweeps skip those terms there (subtracting an exact
// zero changes nothing) and take the full 8 only in the boundary rows.
constexpr int kNarrowFrom = kBand / 2;   // 4

// Each row is one FMA chain ordered oldest to newest, so the newest solution
// value enters last and the recurrence costs one FMA latency per row (a
// separate partial sum for the second-newest term would put an add on that
// path).

// Forward substitution row: b - sum_e L(j, j-8+e) w_e, w_7 the newest x.
template <bool NARROW>
__device__ __forceinline__ double l_row(const double *row, double (&w)[kBand], double b) {
  double v = b;
#pragma unroll
  for (int e = NARROW ? kNarrowFrom : 0; e < kBand; ++e) v -= row[e] * w[e];
#pragma unroll
  for (int e = 0; e < kBand - 1; ++e) w[e] = w[e + 1];
  w[kBand - 1] = v;
  return v;
}

// Backward substitution row with U = D U': b / u_jj - sum_f U'(j, j+f) w_{f-1},
// w_0 the newest x (row[0] = 1/u_jj, row[f] = U'(j, j+f)).
template <bool NARROW>
__device__ __forceinline__ double u_row(const double *row, double (&w)[kBand], double b) {
  double v = b * row[0];
#pragma unroll
  for (int f = NARROW ? kNarrowFrom : kBand; f >= 1; --f) v -= row[f] * w[f - 1];
#pragma unroll
  for (int f = kBand - 1; f > 0; --f) w[f] = w[f - 1];
  w[0] = v;
  return v;
}

// U^T forward row (column-oriented), U^T = U'^T D: z = b - pending_0 solves
// the unit factor, y = z / u_ii, and the pending sums of rows i+1..i+8 take
// U'(i, i+f) z.
template <bool NARROW>
__device__ __forceinline__ double ut_row(const double *row, double (&w)[kBand], double b) {
  const double z = b - w[0];
  constexpr int kn = NARROW ? kNarrowFrom : kBand - 1;
#pragma unroll
  for (int k = 0; k < kn; ++k) w[k] = w[k + 1] + row[k + 1] * z;
#pragma unroll
  for (int k = kn; k < kBand - 1; ++k) w[k] = w[k + 1];
  w[kBand - 1] = NARROW ? 0.0 : row[kBand] * z;
  return z * row[0];
}

// L^T backward row: x = b - pending_0, then the pending sums of rows
// j-1..j-8 take L(j, j-1-k) x.
template <bool NARROW>
__device__ __forceinline__ double lt_row(const double *row, double (&w)[kBand], double b) {
  const double xj = b - w[0];
  constexpr int kn = NARROW ? kNarrowFrom : kBand - 1;
#pragma unroll
  for (int k = 0; k < kn; ++k) w[k] = w[k + 1] + row[kBand - 1 - k] * xj;
#pragma unroll
  for (int k = kn; k < kBand - 1; ++k) w[k] = w[k + 1];
  w[kBand - 1] = NARROW ? 0.0 : row[0] * xj;
  return xj;
}

// TRANS = false: solve A x = b with A = L U (L then U).  TRANS = true: solve
// A^T x = b = U^T L^T x: forward over U rows (column-oriented: after x_i is
// known, its products with row i of U are added to the pending sums of rows
// i+1..i+8), then backward over L rows the same way, so each chunk still only
// needs its own rows of the factors.
// One sweep tile run by the 4 kSweepOps threads tid = 0.. of a group that
// synchronises with sync() (the whole CTA in k_sweep; a named barrier of the
// group in the persistent ensemble kernel).  ring_raw: kSweepSmem bytes of
// shared memory, bars: NST mbarriers, abort_flag: one shared int, all
// private to the group.  NST: depth of the factor ring (NST in
// k_sweep; ring_raw holds NST stages of kSweepStageDoubles).
template <bool TRANS, int NST, typename Sync>
__device__ __forceinline__ void sweep_body(const SweepArgs &a, DevScalars *sc, int bx, int by,
                                           int bz, int tid, double *ring_raw,
                                           unsigned long long *bars, int *abort_flag,
                                           Sync sync) {
  auto ring = [&](int st) { return ring_raw + st * kSweepStageDoubles; };
  const SweepField F = a.f[bz];
  const int m = by;
  const int K1 = a.K + 1;
  const int g0 = bx * kSweepOps;
  const int nops = min(kSweepOps, K1 - g0);
  int q = m + F.qshift;
  if (q < 0) q = -q;
  if (F.qshift < 0 && m == 0) q = 1;
  const int o0 = q * K1 + g0;
  const int g = tid >> 2;
  const int part = tid & 1;
  const int neg = (tid >> 1) & 1;
  const int ak = g0 + g;
  const int kk = neg ? a.NK - ak : ak;
  bool active = (g < nops) && !(neg && ak == 0) && !(F.skip00 && m == 0 && ak == 0);
  // debug build: the system's last row must lie inside its plane
  if (active && !dbg_in((long long)(a.Nr - 1) * a.nmode + (long long)m * a.NK + kk, a.S,
                        DBG_SWEEP_X))
    active = false;
  double *x = F.x + part * a.S + (long long)m * a.NK + (active ? kk : 0);
  const long long xs = a.nmode;
  const int nch = (a.Nr + kSweepRows - 1) / kSweepRows;

  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < NST; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  sync();
  // per-stage bits: current mbarrier phase, and copies in flight (thread 0)
  unsigned phase = 0u, armed = 0u;
  // chunk sequence: forward L chunks 0..nch-1, then backward U chunks nch-1..0
  const int total = 2 * nch;
  auto arm = [&](int step, int s) {
    if (!a.arm) return;
    const bool first = step < nch;   // forward pass
    const int j0 = (first ? step : total - 1 - step) * kSweepRows;
    if (first != TRANS)   // forward of A, or backward of A^T: L rows
      arm_chunk<kBand>(smem_u32(&bars[s]), ring(s), F.L, a.Nrp, o0, nops, j0, F.nop);
    else
      arm_chunk<kBand + 1>(smem_u32(&bars[s]), ring(s), F.U, a.Nrp, o0, nops, j0, F.nop);
    armed |= 1u << s;
  };
  if (tid == 0)
    for (int s = 0; s < NST && s < total; ++s) arm(s, s);

  double w[kBand];
#pragma unroll
  for (int e = 0; e < kBand; ++e) w[e] = 0.0;
  double xa[kSweepRows];
  {
#pragma unroll
    for (int r = 0; r < kSweepRows; ++r) xa[r] = (active && r < a.Nr) ? x[r * xs] : 0.0;
  }
  bool ok = true;
  for (int step = 0; step < total; ++step) {
    const int s = step % NST;
    const bool fwd = step < nch;
    const int c = fwd ? step : total - 1 - step;
    const int j0 = c * kSweepRows;
    if (fwd && step == nch - 1) {
      // backward sweep starts from the chunk just finished: nothing to prefetch
    }
    const bool done = mbar_wait(smem_u32(&bars[s]), (phase >> s) & 1u);
    if (!done) {
      ok = false;
      atomicOr(abort_flag, 1);
    } else {
      phase ^= 1u << s;
      if (tid == 0) armed &= ~(1u << s);   // its copies have landed
    }
    sync();
    if (*abort_flag) break;
    if (active) {
      // The narrow/wide choice is made per chunk (a chunk with any boundary
      // row takes the wide form for all its rows: the extra terms are exact
      // zeros), so a full chunk is straight-line code in which the sliding
      // window w[] lives in renamed registers; only a chunk past the last row
      // guards each row.
      const bool full = j0 + kSweepRows <= a.Nr;
      const bool low_narrow = j0 + kSweepRows <= a.Nr - kNarrowFrom;   // L rows, L^T rows
      const bool up_narrow = j0 >= kNarrowFrom;                        // U rows, U^T rows
      const double *Lc = ring(s) + g * kSweepOpDoubles;                // stage holds L or U
      if (TRANS && fwd) {
        // U^T y = b: z_i = b_i - pending_i, y_i = z_i / u_ii, pending += U'(i, i+f) z_i
        if (full && up_narrow) {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            x[(j0 + r) * xs] = ut_row<true>(Lc + r * (kBand + 1), w, xa[r]);
        } else if (full) {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            x[(j0 + r) * xs] = ut_row<false>(Lc + r * (kBand + 1), w, xa[r]);
        } else {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            if (j0 + r < a.Nr) x[(j0 + r) * xs] = ut_row<false>(Lc + r * (kBand + 1), w, xa[r]);
        }
      } else if (TRANS) {
        // L^T x = y: x_j = y_j - pending_j, then pending_{j-8+e} += L(j, j-8+e) x_j
        if (full && low_narrow) {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            x[(j0 + r) * xs] = lt_row<true>(Lc + r * kBand, w, xa[r]);
        } else if (full) {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            x[(j0 + r) * xs] = lt_row<false>(Lc + r * kBand, w, xa[r]);
        } else {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            if (j0 + r < a.Nr) x[(j0 + r) * xs] = lt_row<false>(Lc + r * kBand, w, xa[r]);
        }
      } else if (fwd) {
        if (full && low_narrow) {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            x[(j0 + r) * xs] = l_row<true>(Lc + r * kBand, w, xa[r]);
        } else if (full) {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            x[(j0 + r) * xs] = l_row<false>(Lc + r * kBand, w, xa[r]);
        } else {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r)
            if (j0 + r < a.Nr) x[(j0 + r) * xs] = l_row<false>(Lc + r * kBand, w, xa[r]);
        }
      } else {
        if (full && up_narrow) {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            x[(j0 + r) * xs] = u_row<true>(Lc + r * (kBand + 1), w, xa[r]);
        } else if (full) {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            x[(j0 + r) * xs] = u_row<false>(Lc + r * (kBand + 1), w, xa[r]);
        } else {
#pragma unroll
          for (int r = kSweepRows - 1; r >= 0; --r)
            if (j0 + r < a.Nr) x[(j0 + r) * xs] = u_row<false>(Lc + r * (kBand + 1), w, xa[r]);
        }
      }
      // prefetch the right-hand sides of the next chunk
      if (fwd) {
        if (c + 1 < nch) {
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r) {
            const int j = j0 + kSweepRows + r;
            xa[r] = (j < a.Nr) ? x[j * xs] : 0.0;
          }
        } else {   // the backward sweep starts from the chunk just finished
#pragma unroll
          for (int e = 0; e < kBand; ++e) w[e] = 0.0;
#pragma unroll
          for (int r = 0; r < kSweepRows; ++r) {
            const int j = j0 + r;
            xa[r] = (j < a.Nr) ? x[j * xs] : 0.0;
          }
        }
      } else if (c > 0) {
#pragma unroll
        for (int r = 0; r < kSweepRows; ++r) xa[r] = x[(j0 - kSweepRows + r) * xs];
      }
    }
    sync();   // every thread is done with stage s
    if (tid == 0 && step + NST < total) arm(step + NST, s);
  }
  if (!ok) atomicOr(&sc->timeout, 1);
  if (*abort_flag && tid == 0) {
    // drain the copies still in flight into this CTA's ring, bounded again
    for (int s = 0; s < NST; ++s)
      if ((armed >> s) & 1u) mbar_wait(smem_u32(&bars[s]), (phase >> s) & 1u);
  }
  // the barriers are invalidated so that their shared memory can be reused
  // (the persistent ensemble kernel runs many tiles in the same CTA)
  sync();
  if (tid == 0)
    for (int s = 0; s < NST; ++s)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(&bars[s])) : "memory");
}

// Influence coefficients per mode: alpha = -Ainv [div u0 (r_i), div u0 (r_o)].
// Two lanes per mode: lane w forms the wall divergence at wall w, the pair
// swaps them, and lane w writes row w of alpha.
__device__ __forceinline__ void alpha_body(const double *__restrict__ U,
                                           double2 *__restrict__ alpha, const LinParams &p,
                                           long long t) {
  const Sizes &s = p.sz;
  const int mode = (int)(t >> 1);
  const int w = (int)(t & 1);
  const bool live = mode < s.nmode && mode != 0;
  const long long S = s.S;
  double2 d = {0.0, 0.0};
  int o = 0;
  if (live) {
    const int m = mode / s.NK, kk = mode % s.NK;
    const int kv = kval(kk, s.K, s.NK);
    o = m * (s.K + 1) + (kv < 0 ? -kv : kv);
    const int j = (w == 0) ? 0 : s.Nr - 1;
    const int st = p.rad.s0[j];
    double2 acc = {0.0, 0.0};
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
      const long long ii = (long long)(st + q) * s.nmode + mode;
      if (!dbg_in(ii, S, DBG_ALPHA)) continue;
      const double2 up = {U[ii], U[S + ii]}, um = {U[2 * S + ii], U[3 * S + ii]};
      const double2 ur = 0.5 * (up + um);
      acc = acc + p.rad.D1[j * kStencil + q] * (p.rad.r[st + q] * ur);
    }
    d = p.rad.inv_r[j] * acc;
  }
  // lanes 2i, 2i+1 hold the two walls of one mode (the grid is whole warps)
  const double ox = __shfl_xor_sync(0xffffffffu, d.x, 1);
  const double oy = __shfl_xor_sync(0xffffffffu, d.y, 1);
  if (!live) return;
  const double2 d0 = w == 0 ? d : double2{ox, oy};
  const double2 d1 = w == 0 ? double2{ox, oy} : d;
  const int nop = p.nopP;
  if (!dbg_in(o, nop, DBG_ALPHA)) return;
  const double a0 = p.Ainv[(2 * w) * nop + o], a1 = p.Ainv[(2 * w + 1) * nop + o];
  alpha[(long long)w * s.nmode + mode] =
      double2{-(a0 * d0.x + a1 * d1.x), -(a0 * d0.y + a1 * d1.y)};
}

// Every thread of the CTA must call it (the corrector difference is reduced
// over the CTA).
__device__ __forceinline__ void correct_body(const double *__restrict__ U,
                                             const double *__restrict__ Ps,
                                             const double2 *__restrict__ alpha,
                                             double2 *__restrict__ Xout,
                                             double2 *__restrict__ Pout,
                                             const double2 *__restrict__ Xprev,
                                             const LinParams &p, DevScalars *sc, long long i) {
  const Sizes &s = p.sz;
  // max |Xout - Xprev| over this thread's coefficients, kept as the bit
  // pattern (non-negative doubles order like their bits), so only the
  // subtractions use the FP64 pipe
  unsigned long long dbits = 0ull;
  if (i < s.S) {
    const int j = (int)i / s.nmode;
    const int mode = (int)(i - (long long)j * s.nmode);
    const long long S = s.S;
    double2 up = {U[i], U[S + i]}, um = {U[2 * S + i], U[3 * S + i]},
            uz = {U[4 * S + i], U[5 * S + i]};
    double2 pr = {0.0, 0.0};
    double2 xr, xt;
    if (mode == 0) {
      xr = {0.0, 0.0};   // u_r = 0; slot 0 holds u_theta
      xt = up;
    } else {
      const int m = mode / s.NK, kk = mode % s.NK;
      const int kv = kval(kk, s.K, s.NK);
      const int o = m * (s.K + 1) + (kv < 0 ? -kv : kv);
      const double beta = p.betak[kk];
      const double2 a = alpha[mode], b = alpha[s.nmode + mode];
      const long long fs = (long long)s.Nr * p.nopP;
      const long long jo = dbg_in(o, p.nopP, DBG_CORRECT) ? (long long)j * p.nopP + o : 0;
      const double *F = p.infl;
      pr = double2{Ps[i], Ps[S + i]};
      pr = pr + F[0 * fs + jo] * a;
      pr = pr + F[1 * fs + jo] * b;
      up = up + F[2 * fs + jo] * a;
      um = um + F[3 * fs + jo] * a;
      up = up + F[4 * fs + jo] * b;
      um = um + F[5 * fs + jo] * b;
      // u_z of a homogeneous solution = -i beta zeta
      uz = uz + (-beta * F[6 * fs + jo]) * mul_i(a);
      uz = uz + (-beta * F[7 * fs + jo]) * mul_i(b);
      xr = 0.5 * (up + um);
      xt = div_2i(up - um);
    }
    Xout[i] = xr;
    Xout[S + i] = xt;
    Xout[2 * S + i] = uz;
    // NaN/Inf test on the exponent bits (integer ops, off the FP64 pipe)
    auto exp_all = [](double2 v) {
      return (__double2hiint(v.x) & 0x7ff00000) == 0x7ff00000 ||
             (__double2hiint(v.y) & 0x7ff00000) == 0x7ff00000;
    };
    bool bad = exp_all(xr) || exp_all(xt) || exp_all(uz);
    double2 T = {0.0, 0.0};
    if (s.nf == 4) {
      T = double2{U[6 * S + i], U[7 * S + i]};
      Xout[3 * S + i] = T;
      bad = bad || exp_all(T);
    }
    if (Pout) Pout[i] = pr;
    if (bad) atomicOr(&sc->nonfinite, 1);
    if (Xprev) {
      auto dm = [&](double2 a, double2 b) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(fabs(a.x - b.x));
        const unsigned long long v = (unsigned long long)__double_as_longlong(fabs(a.y - b.y));
        dbits = max(dbits, max(u, v));
      };
      dm(xr, Xprev[i]);
      dm(xt, Xprev[S + i]);
      dm(uz, Xprev[2 * S + i]);
      if (s.nf == 4) dm(T, Xprev[3 * S + i]);
    }
  }
  if (Xprev) {   // uniform over the grid: every thread of every block gets here
    // the last corrector: X, Yb, N1 and P now belong to one stage
    if (i == 0) sc->rhs_ident = 1;
    __shared__ unsigned long long wmax[32];
    for (int o = 16; o > 0; o >>= 1) dbits = max(dbits, __shfl_xor_sync(0xffffffffu, dbits, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dbits;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) dbits = max(dbits, wmax[w]);
      // one atomic per block, and none once a larger value is in place
      if (dbits > *reinterpret_cast<volatile unsigned long long *>(&sc->corr_bits))
        atomicMax(&sc->corr_bits, dbits);
    }
  }
}

}  // namespace
}  // namespace tc
