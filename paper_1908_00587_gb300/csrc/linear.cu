// Linear stage: per-Fourier-mode radial Helmholtz / Poisson solves.
//
// Paper Sec. 2.2: the Fourier modes are independent in the linear terms (the
// MPI code distributes them in slabs and OpenMP threads loop over them; the
// GPU code uses its own linear-algebra kernels).  Here one thread owns one
// radial system; consecutive threads take consecutive modes, so every load of
// a radial node is coalesced across systems in the [r][m][k] layout.
//
// Scheme (predictor-corrector of Sec. 2.1, Crank-Nicolson weight c = 1/2):
//   R   = X^n/dt + (1-c) L X^n + (1-c) N^n + c N        (N = N^n or N(X*))
//   p0  : L p0 = div R inside, D1 p0 = 0 at both walls
//   u0  : (I/dt - c L+-) u+- = R+- - (D1 p0 -+ (m/r) p0),
//         (I/dt - c L) u_z = R_z - i beta p0, no-slip rows
//   u   = u0 + a_i u_a + a_o u_b with the 2x2 influence matrix chosen so that
//         div u = 0 at both wall nodes (u_a, u_b from unit wall fluxes of p).
// u+- = u_r +- i u_theta decouples the viscous terms:
//   L+- = D2 + D1/r - (m+-1)^2/r^2 - beta^2, L = D2 + D1/r - m^2/r^2 - beta^2.
// The band LU (no pivoting; the operators are diagonally dominant or, for the
// pressure, checked against the pivoted dense solve in the tests) stores 8
// sub-diagonals, the inverse diagonal and 8 super-diagonals per row.
#include <cuda_runtime.h>

#include "lin_body.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

__global__ void k_factor_poisson(LinParams p) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= p.nopP || o == 0) return;   // (0,0) has no pressure solve
  const int m = o / (p.sz.K + 1), ak = o % (p.sz.K + 1);
  const double beta = p.alpha * ak;
  band_factor(p.rad, p.sz.Nr, 0, (double)m * m, beta * beta, 0.0, 0.0, p.LP, p.UP, p.Nrp, o);
}

__global__ void k_factor_helm(LinParams p, const DevScalars *sc) {
  factor_helm_body(p, sc, blockIdx.x * blockDim.x + threadIdx.x);
}

// Homogeneous solutions and the inverse influence matrix, per (m, |k|).
__global__ void k_influence(LinParams p, const DevScalars *sc) {
  influence_body(p, sc, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_dt_policy(DevScalars *sc, double dt_fixed, double cfl, double dt_max,
                            double *dt_hist, int hist_cap) {
  dt_policy_body(sc, dt_fixed, cfl, dt_max, dt_hist, hist_cap);
}

__global__ void k_rhs(const double2 *__restrict__ X, const double2 *__restrict__ N,
                      double2 *__restrict__ Yb, const double2 *__restrict__ N1,
                      const double2 *__restrict__ P, LinParams p, const DevScalars *sc) {
  rhs_body(X, N, Yb, N1, P, p, sc, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(kPrThreads)
k_prhs(const double2 *__restrict__ Yb, const double2 *__restrict__ N, double *__restrict__ Ps,
       double *__restrict__ UT, LinParams p) {
  __shared__ double2 Rr[kPrWin * kPrW];
  prhs_body(Yb, N, Ps, UT, p, Rr, blockIdx.x, blockIdx.y);
}

__global__ void k_hrhs(const double2 *__restrict__ Yb, const double2 *__restrict__ N,
                       const double *__restrict__ Ps, double *__restrict__ U, LinParams p) {
  hrhs_body(Yb, N, Ps, U, p, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};

template <bool TRANS>
__global__ void __launch_bounds__(4 * kSweepOps)
k_sweep(SweepArgs a, DevScalars *sc) {
  extern __shared__ __align__(128) double ring_raw[];
  __shared__ __align__(8) unsigned long long bars[kSweepStages];
  __shared__ int abort_flag;
  sweep_body<TRANS, kSweepStages>(a, sc, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x,
                                  ring_raw, bars, &abort_flag, CtaSync{});
}

__global__ void k_alpha(const double *__restrict__ U, double2 *__restrict__ alpha, LinParams p) {
  alpha_body(U, alpha, p, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_correct(const double *__restrict__ U, const double *__restrict__ Ps,
                          const double2 *__restrict__ alpha, double2 *__restrict__ Xout,
                          double2 *__restrict__ Pout, const double2 *__restrict__ Xprev,
                          LinParams p, DevScalars *sc) {
  correct_body(U, Ps, alpha, Xout, Pout, Xprev, p, sc,
               (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Axial-flux constraint on the (0,0) u_z column (one CTA): the stage's u_z
// gets G times the response ug to a unit uniform forcing (Dirichlet walls),
// G = -Q(u_z) / Q(ug) with Q(f) = sum_j w_j r_j f_j the axial volume flux
// (Clenshaw-Curtis weights), so the flux after the stage is zero.
__global__ void k_flux(double2 *__restrict__ X, const double *__restrict__ ug, LinParams p) {
  const Sizes &s = p.sz;
  __shared__ double red[2][32];
  double q = 0.0, qg = 0.0;
  for (int j = threadIdx.x; j < s.Nr; j += blockDim.x) {
    const double w = p.rad.wr[j];
    q += w * X[2 * s.S + (long long)j * s.nmode].x;
    qg += w * ug[j];
  }
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_xor_sync(0xffffffffu, q, o);
    qg += __shfl_xor_sync(0xffffffffu, qg, o);
  }
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][wid] = q;
    red[1][wid] = qg;
  }
  __syncthreads();
  double Q = 0.0, Qg = 0.0;
  for (int k = 0; k < nw; ++k) {
    Q += red[0][k];
    Qg += red[1][k];
  }
  const double G = -Q / Qg;
  for (int j = threadIdx.x; j < s.Nr; j += blockDim.x)
    X[2 * s.S + (long long)j * s.nmode].x += G * ug[j];
}

// ---------------------------------------------------------------------------
// Adjoint of the implicit stage (its linear part: the wall values are
// constants) and of the explicit right-hand side, in the real Euclidean inner
// product of stored (Re, Im) coefficients.  Transposes, in reverse order:
//   primitive <- +- and influence correction (k_stT_correct, k_stT_alpha),
//   Helmholtz solves (k_sweep<true>), Helmholtz right-hand side with grad p
//   (k_stT_hrhs), Poisson solve (k_sweep<true>), div R (k_stT_prhs).
// Multiplication by a complex constant a transposes to multiplication by
// conj(a); a radial stencil transposes to the gather over the rows whose
// stencil contains the node.

// Lbar (primitive) -> cotangent of u0 in the Helmholtz slots (U planes).
__global__ void k_stT_correct(const double2 *__restrict__ Lb, double *__restrict__ U, Sizes s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.S) return;
  const int mode = (int)(i % s.nmode);
  const long long S = s.S;
  const double2 xr = Lb[i], xt = Lb[S + i], xz = Lb[2 * S + i];
  double2 up, um;
  if (mode == 0) {
    up = xt;                 // slot 0 carries u_theta
    um = double2{0.0, 0.0};
  } else {
    // X_r = (u+ + u-)/2, X_theta = (u+ - u-)/(2i)
    up = double2{0.5 * (xr.x - xt.y), 0.5 * (xr.y + xt.x)};
    um = double2{0.5 * (xr.x + xt.y), 0.5 * (xr.y - xt.x)};
  }
  U[i] = up.x;
  U[S + i] = up.y;
  U[2 * S + i] = um.x;
  U[3 * S + i] = um.y;
  U[4 * S + i] = xz.x;
  U[5 * S + i] = xz.y;
  if (s.nf == 4) {
    const double2 xT = Lb[3 * S + i];
    U[6 * S + i] = xT.x;
    U[7 * S + i] = xT.y;
  }
}

// Per mode: alphabar = <homogeneous solutions, ubar>, dbar = -Ainv^T alphabar,
// then the wall-divergence stencils scatter dbar into ubar0 (this thread owns
// the mode's column).
// A CTA takes kAlW modes (lanes) x kAlR row groups (warps): each thread sums
// its rows' share of the homogeneous-solution products, the row groups are
// reduced in shared memory, and one lane per mode forms the wall
// divergence cotangents and scatters them back through the transposed stencil
// (sequentially per mode: with Nr < 18 the two walls' stencils overlap).
constexpr int kAlW = 8, kAlR = 32;   // 8 modes x 32 row groups: small runs still fill the SMs
__global__ void __launch_bounds__(kAlW * kAlR) k_stT_alpha(double *__restrict__ U, LinParams p) {
  const Sizes &s = p.sz;
  __shared__ double red[kAlR][4][kAlW];
  const int tx = threadIdx.x % kAlW, ty = threadIdx.x / kAlW;
  const int mode = blockIdx.x * kAlW + tx;
  const bool live = mode < s.nmode && mode != 0;
  const long long S = s.S;
  int o = 0;
  double beta = 0.0;
  if (live) {
    const int m = mode / s.NK, kk = mode % s.NK;
    const int kv = kval(kk, s.K, s.NK);
    o = m * (s.K + 1) + (kv < 0 ? -kv : kv);
    beta = p.alpha * kv;
  }
  const long long fs = (long long)s.Nr * p.nopP;
  const double *F = p.infl;
  double2 ab[2] = {{0.0, 0.0}, {0.0, 0.0}};
  if (live) {
    for (int j = ty; j < s.Nr; j += kAlR) {
      const long long ii = (long long)j * s.nmode + mode;
      const long long jo = (long long)j * p.nopP + o;
      const double2 up = {U[ii], U[S + ii]}, um = {U[2 * S + ii], U[3 * S + ii]};
      const double2 uz = {U[4 * S + ii], U[5 * S + ii]};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const double hp = F[(2 + 2 * q) * fs + jo], hm = F[(3 + 2 * q) * fs + jo];
        const double zq = F[(6 + q) * fs + jo];
        // u_z of a homogeneous solution is -i beta zeta: transpose is +i beta zeta
        ab[q].x += hp * up.x + hm * um.x - beta * zq * uz.y;
        ab[q].y += hp * up.y + hm * um.y + beta * zq * uz.x;
      }
    }
  }
  red[ty][0][tx] = ab[0].x;
  red[ty][1][tx] = ab[0].y;
  red[ty][2][tx] = ab[1].x;
  red[ty][3][tx] = ab[1].y;
  __syncthreads();
  if (ty != 0 || !live) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int g = 0; g < kAlR; ++g)
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] += red[g][c][tx];
  ab[0] = double2{v[0], v[1]};
  ab[1] = double2{v[2], v[3]};
  const int nop = p.nopP;
  const double a00 = p.Ainv[o], a01 = p.Ainv[nop + o], a10 = p.Ainv[2 * nop + o],
               a11 = p.Ainv[3 * nop + o];
  const double2 d0 = {-(a00 * ab[0].x + a10 * ab[1].x), -(a00 * ab[0].y + a10 * ab[1].y)};
  const double2 d1 = {-(a01 * ab[0].x + a11 * ab[1].x), -(a01 * ab[0].y + a11 * ab[1].y)};
  for (int w = 0; w < 2; ++w) {
    const int j = (w == 0) ? 0 : s.Nr - 1;
    const int st = p.rad.s0[j];
    const double2 d = (w == 0) ? d0 : d1;
#pragma unroll
    for (int t = 0; t < kStencil; ++t) {
      const double cf = 0.5 * p.rad.inv_r[j] * p.rad.D1[j * kStencil + t] * p.rad.r[st + t];
      const long long ii = (long long)(st + t) * s.nmode + mode;
      U[ii] += cf * d.x;
      U[S + ii] += cf * d.y;
      U[2 * S + ii] += cf * d.x;
      U[3 * S + ii] += cf * d.y;
    }
  }
}

// bbar_H (U planes) -> Rbar (+- form, all slots) and pbar (Ps planes).
__global__ void k_stT_hrhs(const double *__restrict__ U, double2 *__restrict__ Rb,
                           double *__restrict__ Ps, LinParams p) {
  const Sizes &s = p.sz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.S) return;
  const int j = (int)i / s.nmode;
  const int mode = (int)(i - (long long)j * s.nmode);
  const long long S = s.S;
  const bool interior = (j > 0 && j < s.Nr - 1);
  double2 b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    b[c] = (c < s.nf && interior) ? double2{U[(2 * c) * S + i], U[(2 * c + 1) * S + i]}
                                  : double2{0.0, 0.0};
  double2 pb = {0.0, 0.0};
  if (mode == 0) {
    // slot 0 = R_theta = (R+ - R-)/(2i): transpose (i/2) b0, -(i/2) b0
    Rb[i] = double2{-0.5 * b[0].y, 0.5 * b[0].x};
    Rb[S + i] = double2{0.5 * b[0].y, -0.5 * b[0].x};
  } else {
    Rb[i] = b[0];
    Rb[S + i] = b[1];
    const int m = mode / s.NK, kk = mode % s.NK;
    const double beta = p.betak[kk];
    if (interior) {
      const double mr = p.mval[m] * p.rad.inv_r[j];
      // slot0: +(m/r) p, slot1: -(m/r) p, slot2: -i beta p (transpose +i beta)
      pb.x = mr * (b[0].x - b[1].x) - beta * b[2].y;
      pb.y = mr * (b[0].y - b[1].y) + beta * b[2].x;
    }
    // -D1^T (b0 + b1) over the interior rows whose stencil holds node j
    for (int e = 0; e < kTrans; ++e) {
      const int jj = p.rad.tj[j * kTrans + e];
      if (jj < 0) break;
      if (jj < 1 || jj > s.Nr - 2) continue;
      const int t = j - p.rad.s0[jj];
      const double w = p.rad.D1[jj * kStencil + t];
      const long long q = (long long)jj * s.nmode + mode;
      pb.x -= w * (U[q] + U[2 * S + q]);
      pb.y -= w * (U[S + q] + U[3 * S + q]);
    }
  }
  Rb[2 * S + i] = b[2];
  if (s.nf == 4) Rb[3 * S + i] = b[3];
  Ps[i] = pb.x;
  Ps[S + i] = pb.y;
}

// bbar_P (Ps planes) -> Rbar += div^T bbar_P (interior rows only, mode != 0).
__global__ void k_stT_prhs(const double *__restrict__ Ps, double2 *__restrict__ Rb, LinParams p) {
  const Sizes &s = p.sz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.S) return;
  const int sn = (int)i / s.nmode;
  const int mode = (int)(i - (long long)sn * s.nmode);
  if (mode == 0) return;
  const long long S = s.S;
  const int m = mode / s.NK, kk = mode % s.NK;
  const double beta = p.betak[kk];
  double2 rr = {0.0, 0.0}, rt = {0.0, 0.0}, rz = {0.0, 0.0};
  for (int e = 0; e < kTrans; ++e) {
    const int j = p.rad.tj[sn * kTrans + e];
    if (j < 0) break;
    if (j < 1 || j > s.Nr - 2) continue;
    const int t = sn - p.rad.s0[j];
    const double w = p.rad.Dw[j * kStencil + t];
    const long long q = (long long)j * s.nmode + mode;
    rr.x += w * Ps[q];
    rr.y += w * Ps[S + q];
  }
  if (sn > 0 && sn < s.Nr - 1) {
    const double2 bp = {Ps[i], Ps[S + i]};
    const double mr = p.mval[m] * p.rad.inv_r[sn];
    rt = double2{mr * bp.y, -mr * bp.x};        // (-i m / r) bp
    rz = double2{beta * bp.y, -beta * bp.x};    // (-i beta) bp
  }
  // R_r = (R+ + R-)/2, R_theta = (R+ - R-)/(2i)
  double2 a = Rb[i], b = Rb[S + i], z = Rb[2 * S + i];
  a.x += 0.5 * rr.x - 0.5 * rt.y;
  a.y += 0.5 * rr.y + 0.5 * rt.x;
  b.x += 0.5 * rr.x + 0.5 * rt.y;
  b.y += 0.5 * rr.y - 0.5 * rt.x;
  z.x += rz.x;
  z.y += rz.y;
  Rb[i] = a;
  Rb[S + i] = b;
  Rb[2 * S + i] = z;
}

// R = Y' + c N (+- of primitive N): Ybar (+=) Rbar, Nbar (=, primitive) c N+-^T Rbar.
__global__ void k_stT_split(const double2 *__restrict__ Rb, double2 *__restrict__ Yb,
                            double2 *__restrict__ Nb, Sizes s, int accumulate) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.S) return;
  const long long S = s.S;
  const double2 rp = Rb[i], rm = Rb[S + i];
  // N+ = N_r + i N_theta, N- = N_r - i N_theta
  Nb[i] = double2{kCN * (rp.x + rm.x), kCN * (rp.y + rm.y)};
  Nb[S + i] = double2{kCN * (rp.y - rm.y), kCN * (rm.x - rp.x)};
  for (int c = 0; c < s.nf; ++c) {
    const double2 r = Rb[c * S + i];
    if (c >= 2) Nb[c * S + i] = double2{kCN * r.x, kCN * r.y};
    if (accumulate) {
      const double2 y = Yb[c * S + i];
      Yb[c * S + i] = double2{y.x + r.x, y.y + r.y};
    } else {
      Yb[c * S + i] = r;
    }
  }
}

// Adjoint of Y' = X/dt + (1-c) L X + (1-c) N:  Xbar = transposed operator of
// Ybar (primitive), Nbar += (1-c) (N+-)^T Ybar.
__global__ void k_rhsT(const double2 *__restrict__ Yb, double2 *__restrict__ Xb,
                       double2 *__restrict__ Nb, LinParams p, const DevScalars *sc) {
  const Sizes &s = p.sz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.S) return;
  const int sn = (int)i / s.nmode;
  const int mode = (int)(i - (long long)sn * s.nmode);
  const long long S = s.S;
  const int m = mode / s.NK, kk = mode % s.NK;
  const double beta = p.betak[kk];
  const double idt = 1.0 / sc->dt;
  const double om = 1.0 - kCN;
  const double ir = p.rad.inv_r[sn];
  const double b2 = beta * beta, ir2 = ir * ir;
  double2 g[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};   // sum_j (D2 + D1/r_j)[j][sn] Ybar(j)
  for (int e = 0; e < kTrans; ++e) {
    const int j = p.rad.tj[sn * kTrans + e];
    if (j < 0) break;
    const int t = sn - p.rad.s0[j];
    const double w = p.rad.Lw[j * kStencil + t];
    const long long q = (long long)j * s.nmode + mode;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < s.nf) {
        const double2 y = Yb[c * S + q];
        g[c].x += w * y.x;
        g[c].y += w * y.y;
      }
    }
  }
  const double qp = (double)(m + 1) * (m + 1), qm = (double)(m - 1) * (m - 1);
  const double dp = qp * ir2 + b2, dm = qm * ir2 + b2, d0 = (double)m * m * ir2 + b2;
  double2 xb[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (c >= s.nf) continue;
    const double2 y = Yb[c * S + i];
    const double d = (c == 0) ? dp : (c == 1) ? dm : d0;
    const double kap = (c == 3) ? p.kappaT : 1.0;
    xb[c] = double2{idt * y.x + om * kap * (g[c].x - d * y.x),
                    idt * y.y + om * kap * (g[c].y - d * y.y)};
    // Nbar += (1-c) (N+-)^T Ybar
    if (c == 0 || c == 1) {
      const double sg = (c == 0) ? 1.0 : -1.0;
      double2 nr = Nb[i], nt = Nb[S + i];
      nr.x += om * y.x;
      nr.y += om * y.y;
      nt.x += sg * om * y.y;    // (-i sg) y
      nt.y -= sg * om * y.x;
      Nb[i] = nr;
      Nb[S + i] = nt;
    } else {
      double2 n = Nb[c * S + i];
      n.x += om * y.x;
      n.y += om * y.y;
      Nb[c * S + i] = n;
    }
  }
  // X+- = X_r +- i X_theta:  Xbar_r = X+bar + X-bar, Xbar_theta = -i X+bar + i X-bar
  Xb[i] = double2{xb[0].x + xb[1].x, xb[0].y + xb[1].y};
  Xb[S + i] = double2{xb[0].y - xb[1].y, xb[1].x - xb[0].x};
  Xb[2 * S + i] = xb[2];
  if (s.nf == 4) Xb[3 * S + i] = xb[3];
}

// Orthogonal projection onto u(0,-k) = conj u(0,k) (and a real (0,0) entry).
__global__ void k_herm_project(double2 *__restrict__ X, Sizes s) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)s.nf * s.Nr * (s.K + 1);
  if (t >= n) return;
  const int k = (int)(t % (s.K + 1));
  double2 *col = X + (t / (s.K + 1)) * s.nmode;
  if (k == 0) {
    col[0].y = 0.0;
  } else {
    const double2 a = col[k], b = col[s.NK - k];
    const double2 h = {0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
    col[k] = h;
    col[s.NK - k] = double2{h.x, -h.y};
  }
}

// Gradient of E_pert = (1/2) int |u - u_base|^2 dV: V w_j r_j c_m (u - u_base).
__global__ void k_objective_grad(const double2 *__restrict__ X, const double2 *__restrict__ base,
                                 double2 *__restrict__ G, Sizes s, Radial rad, double V) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)s.nf * s.S) return;
  const int c = (int)(i / s.S);
  const long long rem = i - (long long)c * s.S;
  const int j = (int)rem / s.nmode;
  const int mode = (int)(rem - (long long)j * s.nmode);
  if (c >= 3) {
    G[i] = double2{0.0, 0.0};
    return;
  }
  const double w = V * rad.wr[j] * ((mode / s.NK == 0) ? 1.0 : 2.0);
  const double2 x = X[i], b = base[i];
  G[i] = double2{w * (x.x - b.x), w * (x.y - b.y)};
}

__global__ void k_check_finite(const double2 *__restrict__ X, long long n, DevScalars *sc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = X[i];
  if (!(isfinite(v.x) && isfinite(v.y))) atomicOr(&sc->nonfinite, 1);
}

// Largest magnitude, Hermitian defect of the m = 0 column and NaN/Inf of a
// candidate state (tc_set_state), one thread per coefficient.
__global__ void k_state_check(const double2 *__restrict__ X, Sizes s, DevScalars *sc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double amax = 0.0, defect = 0.0;
  bool bad = false;
  if (i < (long long)s.nf * s.S) {
    const double2 v = X[i];
    bad = !(isfinite(v.x) && isfinite(v.y));
    amax = fmax(fabs(v.x), fabs(v.y));
    const long long col = i % s.nmode;     // m * NK + kk
    if (col == 0) {
      defect = fabs(v.y);
    } else if (col <= s.K) {
      const double2 w = X[i - col + (s.NK - col)];
      defect = fmax(fabs(v.x - w.x), fabs(v.y + w.y));
    }
  }
  if (bad) atomicOr(&sc->nonfinite, 1);
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    defect = fmax(defect, __shfl_xor_sync(0xffffffffu, defect, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (amax == amax) atomicMax(&sc->chk_bits[0], (unsigned long long)__double_as_longlong(amax));
    if (defect == defect)
      atomicMax(&sc->chk_bits[1], (unsigned long long)__double_as_longlong(defect));
  }
}

// u(0,-k) = conj(u(0,k)) (k > 0 kept), real (0,0), for every field and node.
__global__ void k_symmetrise(double2 *__restrict__ X, Sizes s) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)s.nf * s.Nr * (s.K + 1);
  if (t >= n) return;
  const int k = (int)(t % (s.K + 1));
  const long long fj = t / (s.K + 1);         // field * Nr + node
  double2 *col = X + fj * s.nmode;            // m = 0 column of that node
  if (k == 0) {
    col[0].y = 0.0;
  } else {
    const double2 v = col[k];
    col[s.NK - k] = double2{v.x, -v.y};
  }
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

SweepArgs sweep_args(const tc_ctx *c) {
  SweepArgs a{};
  a.Nr = c->sz.Nr;
  a.Nrp = c->lin.Nrp;
  a.K = c->sz.K;
  a.NK = c->sz.NK;
  a.nmode = c->sz.nmode;
  a.S = c->sz.S;
  a.arm = c->selftest_no_copy ? 0 : 1;
  return a;
}

}  // namespace

void setup_linear(tc_ctx *c) {
  (void)c;
  allow_smem(k_sweep<false>);
  allow_smem(k_sweep<true>);
}

unsigned debug_word_linear(int clear) {
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

void launch_factor_poisson(tc_ctx *c) {
  LaunchScope ls(c, KFACTH);
  k_factor_poisson<<<blocks(c->lin.nopP, 128), 128, 0, c->stream>>>(c->lin);
}

void launch_refactor(tc_ctx *c) {
  const LinParams &p = c->lin;
  {
    LaunchScope ls(c, KFACTH);
    k_factor_helm<<<blocks(p.nopH + p.nopT, 128), 128, 0, c->stream>>>(p, c->scal);
  }
  LaunchScope ls(c, KINFL);
  k_influence<<<blocks(p.nopP, 128), 128, 0, c->stream>>>(p, c->scal);
}

void launch_dt_policy(tc_ctx *c, double dt_fixed, int step_index) {
  LaunchScope ls(c, KDT);
  k_dt_policy<<<1, 1, 0, c->stream>>>(c->scal, dt_fixed, c->cfl, c->dt_max,
                                       step_index >= 0 ? c->dt_hist : nullptr, c->dt_hist_cap);
}

void launch_rhs(tc_ctx *c, const double2 *X, const double2 *N0) {
  LaunchScope ls(c, KRHS);
  k_rhs<<<blocks(c->sz.S, 128), 128, 0, c->stream>>>(X, N0, c->Yb, c->N1, c->P, c->lin,
                                                      c->scal);
}

void invalidate_rhs_identity(tc_ctx *c) {
  cudaMemsetAsync(reinterpret_cast<char *>(c->scal) + offsetof(DevScalars, rhs_ident), 0,
                  sizeof(int), c->stream);
}

void launch_stage(tc_ctx *c, const double2 *N, double2 *Xout, double2 *Pout,
                  const double2 *Xprev) {
  const Sizes &s = c->sz;
  const LinParams &p = c->lin;
  double *U = reinterpret_cast<double *>(c->U0);
  double *UT = (s.nf == 4) ? U + 6 * s.S : nullptr;
  {
    LaunchScope ls(c, KPRHS);
    k_prhs<<<dim3(blocks(s.nmode, kPrW), blocks(s.Nr, kPrL)), kPrThreads, 0, c->stream>>>(
        c->Yb, N, c->Ps, UT, p);
  }
  {
    // the pressure and (independent of it) the temperature
    LaunchScope ls(c, KPOIS);
    SweepArgs sa = sweep_args(c);
    sa.f[0] = SweepField{p.LP, p.UP, c->Ps, 0, 1, p.nopP};
    if (UT) sa.f[1] = SweepField{p.LT, p.UT, UT, 0, 0, p.nopT};
    k_sweep<false><<<dim3((s.K + kSweepOps) / kSweepOps, s.NM, UT ? 2 : 1), 4 * kSweepOps,
                     kSweepSmem, c->stream>>>(sa, c->scal);
  }
  {
    LaunchScope ls(c, KHRHS);
    k_hrhs<<<blocks(s.S, 128), 128, 0, c->stream>>>(c->Yb, N, c->Ps, U, p);
  }
  {
    LaunchScope ls(c, KHELM);
    SweepArgs sa = sweep_args(c);
    sa.f[0] = SweepField{p.LH, p.UH, U + 0 * s.S, +1, 0, p.nopH};
    sa.f[1] = SweepField{p.LH, p.UH, U + 2 * s.S, -1, 0, p.nopH};
    sa.f[2] = SweepField{p.LH, p.UH, U + 4 * s.S, 0, 0, p.nopH};
    k_sweep<false><<<dim3((s.K + kSweepOps) / kSweepOps, s.NM, 3), 4 * kSweepOps, kSweepSmem,
                     c->stream>>>(sa, c->scal);
  }
  {
    LaunchScope ls(c, KALPHA);
    k_alpha<<<blocks(2LL * s.nmode, 64), 64, 0, c->stream>>>(U, c->alpha_buf, p);
  }
  {
    LaunchScope ls(c, KCORR);
    k_correct<<<blocks(s.S, 128), 128, 0, c->stream>>>(U, c->Ps, c->alpha_buf, Xout, Pout,
                                                        Xprev, p, c->scal);
  }
  if (c->flux) {
    LaunchScope ls(c, KFLUX);
    k_flux<<<1, 256, 0, c->stream>>>(Xout, c->flux_ug, p);
  }
}

void launch_state_check(tc_ctx *c, const double2 *X) {
  LaunchScope ls(c, KCHECK);
  k_state_check<<<blocks((long long)c->sz.nf * c->sz.S, 256), 256, 0, c->stream>>>(X, c->sz,
                                                                                 c->scal);
}

void launch_symmetrise(tc_ctx *c, double2 *X) {
  LaunchScope ls(c, KCHECK);
  k_symmetrise<<<blocks((long long)c->sz.nf * c->sz.Nr * (c->sz.K + 1), 256), 256, 0,
                 c->stream>>>(X, c->sz);
}

// Adjoint of one implicit stage: Lb (primitive cotangent of the stage output)
// -> Rb (cotangent of the +- right-hand side).
void launch_stage_adjoint(tc_ctx *c, const double2 *Lb, double2 *Rb) {
  const Sizes &s = c->sz;
  const LinParams &p = c->lin;
  double *U = reinterpret_cast<double *>(c->U0);
  LaunchScope ls(c, KADJ);
  k_stT_correct<<<blocks(s.S, 128), 128, 0, c->stream>>>(Lb, U, s);
  k_stT_alpha<<<blocks(s.nmode, kAlW), kAlW * kAlR, 0, c->stream>>>(U, p);
  SweepArgs sa = sweep_args(c);
  sa.f[0] = SweepField{p.LH, p.UH, U + 0 * s.S, +1, 0, p.nopH};
  sa.f[1] = SweepField{p.LH, p.UH, U + 2 * s.S, -1, 0, p.nopH};
  sa.f[2] = SweepField{p.LH, p.UH, U + 4 * s.S, 0, 0, p.nopH};
  if (s.nf == 4) sa.f[3] = SweepField{p.LT, p.UT, U + 6 * s.S, 0, 0, p.nopT};
  k_sweep<true><<<dim3((s.K + kSweepOps) / kSweepOps, s.NM, s.nf), 4 * kSweepOps, kSweepSmem,
                  c->stream>>>(sa, c->scal);
  k_stT_hrhs<<<blocks(s.S, 128), 128, 0, c->stream>>>(U, Rb, c->Ps, p);
  SweepArgs sp = sweep_args(c);
  sp.f[0] = SweepField{p.LP, p.UP, c->Ps, 0, 1, p.nopP};
  k_sweep<true><<<dim3((s.K + kSweepOps) / kSweepOps, s.NM, 1), 4 * kSweepOps, kSweepSmem,
                  c->stream>>>(sp, c->scal);
  k_stT_prhs<<<blocks(s.S, 128), 128, 0, c->stream>>>(c->Ps, Rb, p);
  c->launches += 5;
}

void launch_stage_split_adjoint(tc_ctx *c, const double2 *Rb, double2 *Ybar, double2 *Nb,
                                int accumulate) {
  LaunchScope ls(c, KADJ);
  k_stT_split<<<blocks(c->sz.S, 128), 128, 0, c->stream>>>(Rb, Ybar, Nb, c->sz, accumulate);
}

void launch_rhs_adjoint(tc_ctx *c, const double2 *Ybar, double2 *Xb, double2 *Nb) {
  LaunchScope ls(c, KADJ);
  k_rhsT<<<blocks(c->sz.S, 128), 128, 0, c->stream>>>(Ybar, Xb, Nb, c->lin, c->scal);
}

void launch_herm_project(tc_ctx *c, double2 *X) {
  LaunchScope ls(c, KADJ);
  k_herm_project<<<blocks((long long)c->sz.nf * c->sz.Nr * (c->sz.K + 1), 256), 256, 0,
                   c->stream>>>(X, c->sz);
}

void launch_objective_grad(tc_ctx *c, const double2 *X, double2 *G) {
  LaunchScope ls(c, KADJ);
  k_objective_grad<<<blocks((long long)c->sz.nf * c->sz.S, 256), 256, 0, c->stream>>>(
      X, c->base_dev, G, c->sz, c->nl.rad, 2.0 * 3.14159265358979323846 * c->Lz);
}

void launch_check_finite(tc_ctx *c, const double2 *X, long long n) {
  k_check_finite<<<blocks(n, 256), 256, 0, c->stream>>>(X, n, c->scal);
}

}  // namespace tc
