// Host side of libtc: validation, radial tables, device memory, the step loop
// and the C ABI entry points declared in include/tc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tc_internal.h"

using cplx = std::complex<double>;

namespace tc {

const char *const kKernelNames[KNUM] = {
    "k_zinv", "k_theta", "k_zfwd", "k_dt_policy", "k_factor", "k_influence",
    "k_rhs", "k_prhs", "k_psolve", "k_hrhs", "k_hsolve", "k_alpha", "k_correct", "k_diag", "k_check",
    "k_flux", "k_regrid", "k_adjoint", "k_theta_tc", "k_zinv_tc"};

LaunchScope::LaunchScope(tc_ctx *c_, int id_) : c(c_), id(id_) {
  c->launches++;
  KernelTimer &t = c->timers[id];
  t.launches++;
  if (!c->timing || c->capturing) return;
  if ((int)t.ev.size() < 2 * (t.used + 1)) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    t.ev.push_back(a);
    t.ev.push_back(b);
  }
  cudaEventRecord(t.ev[2 * t.used], c->stream);
}

LaunchScope::~LaunchScope() {
  if (!c->timing || c->capturing) return;
  KernelTimer &t = c->timers[id];
  cudaEventRecord(t.ev[2 * t.used + 1], c->stream);
  t.used++;
}

// All kernels of one predictor-corrector step, enqueued on the context's
// stream with no host synchronisation (so that a graph can capture it).
// step_index >= 0 records the step used into the step history (next slot of
// a device-side counter that tc_step resets); -1 records nothing.
// One step: predictor, then n_corr correctors on the same explicit part.
// The iterates alternate between X and Xp so that the last one lands in X
// (the predictor may overwrite X: everything that reads X^n -- the first
// nonlinear evaluation, the CFL rate and the explicit part Yb -- comes first).
// The last corrector records max |X_corr - X_prev| for tc_diagnostics.
void enqueue_step(tc_ctx *c, double dt_fixed, int step_index) {
  launch_nonlinear(c, c->X, c->N0, &c->scal->rate_bits, 0);
  launch_dt_policy(c, dt_fixed, step_index);
  launch_refactor(c);
  launch_rhs(c, c->X, c->N0);
  double2 *cur = (c->n_corr % 2) ? c->Xp : c->X;
  launch_stage(c, c->N0, cur, c->P);
  for (int i = 0; i < c->n_corr; ++i) {
    double2 *next = (cur == c->X) ? c->Xp : c->X;
    launch_nonlinear(c, cur, c->N1, nullptr, 0);
    launch_stage(c, c->N1, next, c->P, i + 1 == c->n_corr ? cur : nullptr);
    cur = next;
  }
}

FFTPlan make_plan(int n) {
  FFTPlan p{};
  p.n = n;
  int e2 = 0, m = n;
  while (m % 2 == 0) {
    m /= 2;
    ++e2;
  }
  std::vector<int> rs;
  // as many radix-8 passes as possible; a remainder of 2^1 is folded into two
  // radix-4 passes when that is possible (cheaper than a radix-2 pass)
  int n8 = e2 / 3, rem = e2 % 3;
  if (rem == 1 && n8 >= 1) {
    --n8;
    rs.push_back(4);
    rs.push_back(4);
  } else if (rem == 1) {
    rs.push_back(2);
  } else if (rem == 2) {
    rs.push_back(4);
  }
  for (int i = 0; i < n8; ++i) rs.insert(rs.begin(), 8);
  while (m % 3 == 0) {
    rs.push_back(3);
    m /= 3;
  }
  while (m % 5 == 0) {
    rs.push_back(5);
    m /= 5;
  }
  p.npass = (int)rs.size();
  int Ns = 1, off = 0;
  for (int i = 0; i < p.npass; ++i) {
    p.radix[i] = rs[i];
    p.tw_off[i] = off;
    if (Ns > 1) off += (rs[i] - 1) * Ns;
    p.div_nb[i] = make_fastdiv((unsigned)(n / rs[i]));
    p.div_ns[i] = make_fastdiv((unsigned)Ns);
    Ns *= rs[i];
  }
  return p;
}

FastDiv make_fastdiv(unsigned d) {
  int l = 0;   // ceil(log2 d)
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l - 1 > 0 ? l - 1 : 0;
  return f;
}

// Finite-difference weights at x0 on nodes x[0..n-1] for derivatives 0..2
// (Fornberg, Math. Comp. 51 (1988): weights of the Lagrange interpolant's
// derivatives, built by adding one node at a time).
void fd_weights(double x0, const double *x, int n, double w[3][kStencil]) {
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < n; ++j) w[d][j] = 0.0;
  w[0][0] = 1.0;
  double c1 = 1.0, c4 = x[0] - x0;
  for (int i = 1; i < n; ++i) {
    const int mn = std::min(i, 2);
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i] - x0;
    for (int j = 0; j < i; ++j) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int d = mn; d >= 1; --d) w[d][i] = c1 * (d * w[d - 1][i - 1] - c5 * w[d][i - 1]) / c2;
        w[0][i] = -c1 * c5 * w[0][i - 1] / c2;
      }
      for (int d = mn; d >= 1; --d) w[d][j] = (c4 * w[d][j] - d * w[d - 1][j]) / c3;
      w[0][j] = c4 * w[0][j] / c3;
    }
    c1 = c2;
  }
}

// Pass-major twiddles of a plan, each exp(-2 pi i t / n) with t = q k n/(Ns R)
// evaluated in long double.
void fill_plan_twiddles(const FFTPlan &pl, double2 *out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int n = pl.n;
  for (int i = 0; i < n; ++i) out[i] = double2{0.0, 0.0};
  // w = exp(-i a) as (cos a, -sin a), or in cosine-tangent form (c, t) with
  // w = c (1 + i t); |c| is kept >= 2^-60 so that t is finite (the product
  // c t still rounds to -sin a)
  auto angle = [&](long long q) { return 2.0L * pi * (long double)(q % n) / (long double)n; };
  auto ct = [](long double a) {
    long double c = cosl(a);
    const long double lo = 8.6736173798840354720596224069595337e-19L;   // 2^-60
    if (fabsl(c) < lo) c = c < 0 ? -lo : lo;
    return double2{(double)c, (double)(-sinl(a) / c)};
  };
  int Ns = 1;
  for (int p = 0; p < pl.npass; ++p) {
    const int R = pl.radix[p];
    double2 *o = out + pl.tw_off[p];
    if (Ns > 1) {
      const int step = n / (Ns * R);
      for (int k = 0; k < Ns; ++k) {
        const long long e = (long long)k * step;
        if (R == 4) {            // w, w^2
          o[k] = ct(angle(e));
          o[Ns + k] = ct(angle(2 * e));
        } else if (R == 8) {     // w^4, w, w^2, g = w exp(-i pi/4), g^2
          o[k] = ct(angle(4 * e));
          o[Ns + k] = ct(angle(e));
          o[2 * Ns + k] = ct(angle(2 * e));
          o[3 * Ns + k] = ct(angle(e) + pi / 4);
          o[4 * Ns + k] = ct(angle(2 * e) + pi / 2);
        } else {
          for (int q = 1; q < R; ++q) {
            const long double a = angle(q * e);
            o[(q - 1) * Ns + k] = double2{(double)cosl(a), (double)(-sinl(a))};
          }
        }
      }
    }
    Ns *= R;
  }
}

namespace {

bool smooth235(int n) {
  if (n < 1) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

// Clenshaw-Curtis weights on N+1 Chebyshev-Gauss-Lobatto points of [-1, 1]:
// w_j = (c_j/N) (1 - sum_{k=1}^{N/2} b_k cos(2 k j pi / N) / (4k^2 - 1)),
// c_j = 1 at the ends and 2 inside, b_k = 1 for k = N/2 and 2 otherwise.
std::vector<double> cc_weights(int Nr) {
  const int N = Nr - 1;
  std::vector<double> w(Nr);
  for (int j = 0; j <= N; ++j) {
    long double s = 1.0L;
    for (int k = 1; k <= N / 2; ++k) {
      const long double b = (2 * k == N) ? 1.0L : 2.0L;
      const long long arg = (2LL * k * j) % (2LL * N);
      s -= b * cosl(3.141592653589793238462643383279502884L * (long double)arg / (long double)N) /
           (4.0L * k * k - 1.0L);
    }
    const long double cj = (j == 0 || j == N) ? 1.0L : 2.0L;
    w[j] = (double)(cj / N * s);
  }
  return w;
}

// Dense solve with partial pivoting (set-up only: basic state).
std::vector<double> dense_solve(std::vector<double> A, std::vector<double> b, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] / A[k * n + k];
      if (l == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  std::vector<double> x(n);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return x;
}

std::vector<double2> twiddles(const FFTPlan &pl) {
  std::vector<double2> t(pl.n);
  fill_plan_twiddles(pl, t.data());
  return t;
}

struct CudaError {
  cudaError_t e;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaError{e};
}

template <typename T>
T *dalloc(tc_ctx *c, size_t count) {
  void *p = nullptr;
  const size_t bytes = count * sizeof(T);
  if (over_budget(c, bytes)) throw std::bad_alloc();
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  c->allocs.push_back(p);
  c->device_bytes += bytes;
  return static_cast<T *>(p);
}

// L(q) restricted to (m,k) = (0,0) with Dirichlet rows: dense Nr x Nr.
std::vector<double> dense_lap00(const tc_ctx *c, double q) {
  const int Nr = c->sz.Nr;
  std::vector<double> A((size_t)Nr * Nr, 0.0);
  for (int j = 0; j < Nr; ++j) {
    if (j == 0 || j == Nr - 1) {
      A[(size_t)j * Nr + j] = 1.0;
      continue;
    }
    const int st = c->s0[j];
    for (int t = 0; t < kStencil; ++t)
      A[(size_t)j * Nr + st + t] = c->D2[j * kStencil + t] + c->D1[j * kStencil + t] / c->r[j];
    A[(size_t)j * Nr + j] -= q * q / (c->r[j] * c->r[j]);
  }
  return A;
}

tc_status fail_cuda(tc_ctx *c, cudaError_t e) {
  if (c) c->poisoned = true;
  std::fprintf(stderr, "libtc: CUDA error %s\n", cudaGetErrorString(e));
  return TC_ERR_CUDA;
}

void build_tables(tc_ctx *c) {
  const int Nr = c->sz.Nr;
  c->r.resize(Nr);
  for (int j = 0; j < Nr; ++j)
    c->r[j] = c->r_i + 0.5 * (1.0 - std::cos(M_PI * (double)j / (double)(Nr - 1)));
  c->D1.assign((size_t)Nr * kStencil, 0.0);
  c->D2.assign((size_t)Nr * kStencil, 0.0);
  c->s0.resize(Nr);
  for (int j = 0; j < Nr; ++j) {
    const int st = std::min(std::max(j - kStencil / 2, 0), Nr - kStencil);
    c->s0[j] = st;
    double w[3][kStencil];
    fd_weights(c->r[j], &c->r[st], kStencil, w);
    for (int t = 0; t < kStencil; ++t) {
      c->D1[j * kStencil + t] = w[1][t];
      c->D2[j * kStencil + t] = w[2][t];
    }
  }
  std::vector<double> cc = cc_weights(Nr);
  c->w.resize(Nr);
  c->dr_min.resize(Nr);
  for (int j = 0; j < Nr; ++j) {
    c->w[j] = 0.5 * cc[j];
    const double lo = j > 0 ? c->r[j] - c->r[j - 1] : 1e300;
    const double hi = j < Nr - 1 ? c->r[j + 1] - c->r[j] : 1e300;
    c->dr_min[j] = std::min(lo, hi);
  }
}

void build_base(tc_ctx *c) {
  const int Nr = c->sz.Nr;
  const long long S = c->sz.S;
  c->base.assign((size_t)2 * c->sz.nf * S, 0.0);
  auto put = [&](int f, const std::vector<double> &prof) {
    for (int j = 0; j < Nr; ++j) c->base[2 * ((size_t)f * S + (size_t)j * c->sz.nmode)] = prof[j];
  };
  std::vector<double> b(Nr, 0.0);
  b[0] = c->Re_i;
  b[Nr - 1] = c->Re_o;
  put(1, dense_solve(dense_lap00(c, 1.0), b, Nr));
  c->Tb_disc.assign(Nr, 0.0);
  if (c->has_T) {
    std::fill(b.begin(), b.end(), 0.0);
    b[0] = 0.5;
    b[Nr - 1] = -0.5;
    c->Tb_disc = dense_solve(dense_lap00(c, 0.0), b, Nr);
    put(3, c->Tb_disc);
    for (int j = 0; j < Nr; ++j) b[j] = -c->Gr * c->Tb_disc[j];
    b[0] = 0.0;
    b[Nr - 1] = 0.0;
    std::vector<double> uz = dense_solve(dense_lap00(c, 0.0), b, Nr);
    if (c->flux) {
      // zero axial flux: L(0) u_z = -Gr T - G, G from the response to -1
      std::vector<double> one(Nr, -1.0);
      one[0] = 0.0;
      one[Nr - 1] = 0.0;
      const std::vector<double> uc = dense_solve(dense_lap00(c, 0.0), one, Nr);
      double q = 0.0, qc = 0.0;
      for (int j = 0; j < Nr; ++j) {
        q += c->w[j] * c->r[j] * uz[j];
        qc += c->w[j] * c->r[j] * uc[j];
      }
      for (int j = 0; j < Nr; ++j) uz[j] -= (q / qc) * uc[j];
    }
    put(2, uz);
  }
}

void allocate(tc_ctx *c) {
  const Sizes &s = c->sz;
  const long long S = s.S;
  const int nf = s.nf;
  c->X = dalloc<double2>(c, (size_t)nf * S);
  c->Xp = dalloc<double2>(c, (size_t)nf * S);
  c->N0 = dalloc<double2>(c, (size_t)nf * S);
  c->N1 = dalloc<double2>(c, (size_t)nf * S);
  c->Yb = dalloc<double2>(c, (size_t)nf * S);
  c->U0 = dalloc<double2>(c, (size_t)nf * S);
  c->P = dalloc<double2>(c, (size_t)S);
  c->Ps = dalloc<double>(c, (size_t)2 * S);
  c->base_dev = dalloc<double2>(c, (size_t)nf * S);
  c->alpha_buf = dalloc<double2>(c, (size_t)2 * s.nmode);
  c->V = dalloc<double2>(c, (size_t)3 * nf * s.Nr * s.Nz * s.NM);
  c->W = dalloc<double2>(c, (size_t)nf * s.Nr * s.Nz * s.NM);
  c->prof = dalloc<double>(c, (size_t)8 * s.Nr);
  c->d_r = dalloc<double>(c, s.Nr);
  c->d_inv_r = dalloc<double>(c, s.Nr);
  c->d_D1 = dalloc<double>(c, (size_t)s.Nr * kStencil);
  c->d_D2 = dalloc<double>(c, (size_t)s.Nr * kStencil);
  c->d_Lw = dalloc<double>(c, (size_t)s.Nr * kStencil);
  c->d_Dw = dalloc<double>(c, (size_t)s.Nr * kStencil);
  c->d_tj = dalloc<int>(c, (size_t)s.Nr * kTrans);
  c->d_dr = dalloc<double>(c, s.Nr);
  c->d_cflinv = dalloc<double>(c, (size_t)2 * s.Nr);
  c->d_wr = dalloc<double>(c, s.Nr);
  c->d_s0 = dalloc<int>(c, s.Nr);
  c->d_twz = dalloc<double2>(c, s.Nz);
  c->d_twt = dalloc<double2>(c, s.Nt);
  c->d_f32 = dalloc<float>(c, (size_t)2 * s.Nz + 2 * s.Nt + (size_t)kStencil * s.Nr + s.NK + s.Nr);
  c->d_prof32 = dalloc<float>(c, (size_t)2 * s.Nr);
  c->d_kmtab = dalloc<double>(c, (size_t)s.NK + s.NM);
  const int K1 = s.K + 1;
  c->lin.nopP = s.NM * K1;
  c->lin.nopH = (s.NM + 1) * K1;
  c->lin.nopT = c->has_T ? s.NM * K1 : 0;
  const int Nrp = (s.Nr + kSweepRows - 1) / kSweepRows * kSweepRows;
  c->lin.Nrp = Nrp;
  auto band = [&](int nop, double **L, double **U) {
    *L = dalloc<double>(c, (size_t)std::max(nop, 1) * Nrp * kBand);
    *U = dalloc<double>(c, (size_t)std::max(nop, 1) * Nrp * (kBand + 1));
    ck(cudaMemset(*L, 0, sizeof(double) * std::max(nop, 1) * Nrp * kBand));
    ck(cudaMemset(*U, 0, sizeof(double) * std::max(nop, 1) * Nrp * (kBand + 1)));
  };
  band(c->lin.nopP, &c->LP, &c->UP);
  band(c->lin.nopH, &c->LH, &c->UH);
  band(c->lin.nopT, &c->LT, &c->UT);
  c->infl = dalloc<double>(c, (size_t)8 * s.Nr * c->lin.nopP);
  c->Ainv = dalloc<double>(c, (size_t)4 * c->lin.nopP);
  c->diag_part = dalloc<double>(c, (size_t)s.Nr * 7);
  c->diag_out = dalloc<double>(c, 16);
  {
    static_assert(sizeof(DevScalars) <= tc_ctx::kPinnedScal, "scalars fit their slot");
    unsigned char *blk =
        dalloc<unsigned char>(c, tc_ctx::kPinnedScal + sizeof(double) * tc_ctx::kPinnedHist);
    c->scal = reinterpret_cast<DevScalars *>(blk);
    c->dt_hist = reinterpret_cast<double *>(blk + tc_ctx::kPinnedScal);
    c->dt_hist_cap = tc_ctx::kPinnedHist;
    c->dt_hist_own = false;
  }
  ck(cudaHostAlloc(reinterpret_cast<void **>(&c->h_step),
                   tc_ctx::kPinnedScal + sizeof(double) * tc_ctx::kPinnedHist,
                   cudaHostAllocDefault));
}

void upload_tables(tc_ctx *c) {
  const Sizes &s = c->sz;
  std::vector<double> inv_r(s.Nr), wr(s.Nr);
  for (int j = 0; j < s.Nr; ++j) {
    inv_r[j] = 1.0 / c->r[j];
    wr[j] = c->w[j] * c->r[j];
  }
  ck(cudaMemcpy(c->d_r, c->r.data(), s.Nr * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_inv_r, inv_r.data(), s.Nr * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_D1, c->D1.data(), c->D1.size() * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_D2, c->D2.data(), c->D2.size() * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_dr, c->dr_min.data(), s.Nr * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_wr, wr.data(), s.Nr * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_s0, c->s0.data(), s.Nr * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<double2> tz = twiddles(make_plan(s.Nz)), tt = twiddles(make_plan(s.Nt));
  ck(cudaMemcpy(c->d_twz, tz.data(), s.Nz * sizeof(double2), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_twt, tt.data(), s.Nt * sizeof(double2), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->diag_part + (size_t)s.Nr * 6, c->Tb_disc.data(), s.Nr * sizeof(double),
                cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->base_dev, c->base.data(), c->base.size() * sizeof(double),
                cudaMemcpyHostToDevice));
  DevScalars sc{};
  ck(cudaMemcpy(c->scal, &sc, sizeof(sc), cudaMemcpyHostToDevice));
  std::vector<double> Lw((size_t)s.Nr * kStencil), Dw((size_t)s.Nr * kStencil);
  for (int j = 0; j < s.Nr; ++j)
    for (int t = 0; t < kStencil; ++t) {
      const size_t q = (size_t)j * kStencil + t;
      Lw[q] = c->D2[q] + c->D1[q] * inv_r[j];
      Dw[q] = inv_r[j] * (c->D1[q] * c->r[c->s0[j] + t]);
    }
  ck(cudaMemcpy(c->d_Lw, Lw.data(), Lw.size() * sizeof(double), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(c->d_Dw, Dw.data(), Dw.size() * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<int> tj((size_t)s.Nr * kTrans, -1);
  for (int n = 0; n < s.Nr; ++n) {
    int k = 0;
    for (int j = 0; j < s.Nr; ++j)
      if (c->s0[j] <= n && n < c->s0[j] + kStencil) {
        if (k < kTrans) tj[(size_t)n * kTrans + k] = j;
        ++k;
      }
    if (k > kTrans) throw CudaError{cudaErrorInvalidValue};   // cannot happen (at most 17)
  }
  ck(cudaMemcpy(c->d_tj, tj.data(), tj.size() * sizeof(int), cudaMemcpyHostToDevice));
  Radial rad{c->d_r,  c->d_inv_r, c->d_D1, c->d_D2, c->d_dr,
             c->d_wr, c->d_s0,    c->d_Lw, c->d_Dw, c->d_tj};
  NLParams &p = c->nl;
  p.sz = s;
  p.rad = rad;
  p.alpha = 2.0 * M_PI / c->Lz;
  p.Gr = c->Gr;
  p.dth = 2.0 * M_PI / s.Nt;
  p.dz = c->Lz / s.Nz;
  p.inv_dz = 1.0 / p.dz;
  {
    std::vector<double> ci((size_t)2 * s.Nr);
    for (int j = 0; j < s.Nr; ++j) {
      ci[2 * j] = 1.0 / c->dr_min[j];
      ci[2 * j + 1] = 1.0 / (c->r[j] * p.dth);
    }
    ck(cudaMemcpy(c->d_cflinv, ci.data(), ci.size() * sizeof(double), cudaMemcpyHostToDevice));
    p.cfl_inv = c->d_cflinv;
  }
  p.zscale = 0.5 / ((double)s.Nt * (double)s.Nz);
  p.pz = make_plan(s.Nz);
  p.pt = make_plan(s.Nt);
  p.twz = c->d_twz;
  p.twt = c->d_twt;
  {
    // FP32 tables: twiddles (z, theta), d/dr weights, beta per stored k, 1/r
    std::vector<float> f((size_t)2 * s.Nz + 2 * s.Nt + (size_t)kStencil * s.Nr + s.NK + s.Nr);
    size_t o = 0;
    for (int i = 0; i < s.Nz; ++i) {
      f[o++] = (float)tz[i].x;
      f[o++] = (float)tz[i].y;
    }
    for (int i = 0; i < s.Nt; ++i) {
      f[o++] = (float)tt[i].x;
      f[o++] = (float)tt[i].y;
    }
    const size_t od1 = o;
    for (size_t q = 0; q < (size_t)kStencil * s.Nr; ++q) f[o++] = (float)c->D1[q];
    const size_t obeta = o;
    for (int kk = 0; kk < s.NK; ++kk) f[o++] = (float)(p.alpha * (kk <= s.K ? kk : kk - s.NK));
    const size_t oir = o;
    for (int j = 0; j < s.Nr; ++j) f[o++] = (float)inv_r[j];
    ck(cudaMemcpy(c->d_f32, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    p.twz32 = reinterpret_cast<const float2 *>(c->d_f32);
    p.twt32 = reinterpret_cast<const float2 *>(c->d_f32 + 2 * s.Nz);
    p.d1_32 = c->d_f32 + od1;
    p.beta32 = c->d_f32 + obeta;
    p.inv_r32 = c->d_f32 + oir;
    p.prof32 = c->d_prof32;
  }
  LinParams &l = c->lin;
  l.sz = s;
  l.rad = rad;
  l.alpha = p.alpha;
  l.kappaT = c->has_T ? 1.0 / c->Pr : 1.0;
  l.Re_i = c->Re_i;
  l.Re_o = c->Re_o;
  l.LP = c->LP;
  l.UP = c->UP;
  l.LH = c->LH;
  l.UH = c->UH;
  l.LT = c->LT;
  l.UT = c->UT;
  l.infl = c->infl;
  l.Ainv = c->Ainv;
  {
    std::vector<double> km((size_t)s.NK + s.NM);
    for (int kk = 0; kk < s.NK; ++kk) km[kk] = p.alpha * (double)(kk <= s.K ? kk : kk - s.NK);
    for (int m = 0; m < s.NM; ++m) km[s.NK + m] = (double)m;
    ck(cudaMemcpy(c->d_kmtab, km.data(), km.size() * sizeof(double), cudaMemcpyHostToDevice));
    l.betak = c->d_kmtab;
    l.mval = c->d_kmtab + s.NK;
    p.betak = c->d_kmtab;
  }
}

}  // namespace

// Validate the state staged in Xp (finite, Hermitian m = 0 column within
// 1e-12 of its largest entry), symmetrise it and make it the current state.
// Forgets the dynamic-step history and the flags; the factors stay valid for
// the step they were built for.
tc_status commit_staged_state(tc_ctx *c) {
  const size_t bytes = (size_t)16 * c->sz.nf * c->sz.S;
  try {
    invalidate_rhs_identity(c);
    DevScalars sc{};
    char *base = reinterpret_cast<char *>(c->scal);
    ck(cudaMemsetAsync(base + offsetof(DevScalars, dt_prev), 0, sizeof(double), c->stream));
    ck(cudaMemsetAsync(base + offsetof(DevScalars, rate_bits), 0,
                       offsetof(DevScalars, rate_last) - offsetof(DevScalars, rate_bits),
                       c->stream));
    ck(cudaMemsetAsync(base + offsetof(DevScalars, nonfinite), 0, sizeof(int), c->stream));
    launch_state_check(c, c->Xp);
    ck(cudaGetLastError());
    // the check's verdict through the context's pinned buffer (asynchronous copy)
    ck(cudaMemcpyAsync(c->h_step, c->scal, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    std::memcpy(&sc, c->h_step, sizeof(sc));
    if (sc.nonfinite) return TC_ERR_NONFINITE;
    double amax, defect;
    std::memcpy(&amax, &sc.chk_bits[0], sizeof(double));
    std::memcpy(&defect, &sc.chk_bits[1], sizeof(double));
    if (defect > 1e-12 * amax) return TC_ERR_STATE;
    launch_symmetrise(c, c->Xp);
    ck(cudaMemcpyAsync(c->X, c->Xp, bytes, cudaMemcpyDeviceToDevice, c->stream));
    ck(cudaGetLastError());
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  c->t = 0.0;
  return TC_OK;
}

// Capture one step into a CUDA graph, or keep the one captured before if
// nothing it depends on has changed: the launch parameters (generation
// counter, bumped by every option change and buffer reallocation) and the
// fixed step.  The capture runs on a private stream (the caller's may be the
// legacy default stream, which cannot be captured); the graph is then
// launched on the context's stream.
cudaError_t ensure_step_graph(tc_ctx *c, double dt_fixed) {
  if (c->step_exec && c->graph_gen == c->gen && c->graph_dt == dt_fixed) return cudaSuccess;
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_graph) cudaGraphDestroy(c->step_graph);
  c->step_exec = nullptr;
  c->step_graph = nullptr;
  cudaError_t e = cudaSuccess;
  if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  // the capture stream must not run ahead of work already queued
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  cudaStream_t user = c->stream;
  const long long l0 = c->launches;
  c->stream = c->cap_stream;
  c->capturing = 1;
  e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_step(c, dt_fixed, 0);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    c->step_graph = g;
  }
  c->capturing = 0;
  c->stream = user;
  c->graph_launches = c->launches - l0;
  c->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_exec, c->step_graph, 0);
  if (e != cudaSuccess) return e;
  c->graph_gen = c->gen;
  c->graph_dt = dt_fixed;
  return cudaSuccess;
}


// Capture `enqueue` (kernels and device copies on c->stream) into cg, or keep
// the graph captured before for the same key; then launch it on c->stream.
// Direct launches when timing is on, graphs are off, or the capture fails.
template <typename F>
void run_cached(tc_ctx *c, tc_ctx::CachedGraph &cg, const void *a, const void *b, int n,
                double dt, F enqueue) {
  if (!c->use_graph || c->timing) {
    enqueue();
    return;
  }
  const bool same = cg.exec && cg.gen == c->gen && cg.a == a && cg.b == b && cg.n == n &&
                    cg.dt == dt;
  if (!same) {
    if (cg.exec) cudaGraphExecDestroy(cg.exec);
    if (cg.g) cudaGraphDestroy(cg.g);
    cg.exec = nullptr;
    cg.g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
      cudaStream_t user = c->stream;
      const long long l0 = c->launches;
      c->stream = c->cap_stream;
      c->capturing = 1;
      e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        enqueue();
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        cg.g = g;
      }
      c->capturing = 0;
      c->stream = user;
      cg.launches = c->launches - l0;
      c->launches = l0;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&cg.exec, cg.g, 0);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (cg.g) cudaGraphDestroy(cg.g);
      cg.g = nullptr;
      cg.exec = nullptr;
      enqueue();
      return;
    }
    cg.gen = c->gen;
    cg.a = a;
    cg.b = b;
    cg.n = n;
    cg.dt = dt;
  }
  ck(cudaGraphLaunch(cg.exec, c->stream));
  c->launches += cg.launches;
}

}  // namespace tc

using namespace tc;

extern "C" {

const char *tc_status_string(tc_status s) {
  switch (s) {
    case TC_OK: return "ok";
    case TC_ERR_ARG: return "invalid argument";
    case TC_ERR_CUDA: return "CUDA error (context poisoned)";
    case TC_ERR_OOM: return "out of device memory";
    case TC_ERR_NONFINITE: return "non-finite value in the state";
    case TC_ERR_CFL: return "CFL limit exceeded";
    case TC_ERR_STATE: return "state violates the m = 0 Hermitian symmetry";
    case TC_ERR_TIMEOUT: return "device wait timed out";
    case TC_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

tc_status tc_create(int Nr, int Ntheta, int Nz, double eta, double Lz, double Re_i, double Re_o,
                    double Ra, double Pr, tc_ctx **out) {
  if (!out) return TC_ERR_ARG;
  *out = nullptr;
  if (Nr < kStencil || Nr > 1024) return TC_ERR_ARG;
  if (Ntheta < 4 || Ntheta % 2 != 0 || Nz < 4 || Ntheta > 1024 || Nz > 1024) return TC_ERR_ARG;
  if (!smooth235(Ntheta) || !smooth235(Nz)) return TC_ERR_ARG;
  if (!(eta > 0.0 && eta < 1.0) || !(Lz > 0.0) || !std::isfinite(Lz)) return TC_ERR_ARG;
  if (!std::isfinite(Re_i) || !std::isfinite(Re_o) || !std::isfinite(Ra)) return TC_ERR_ARG;
  if (Ra != 0.0 && !(Pr > 0.0 && std::isfinite(Pr))) return TC_ERR_ARG;
  tc_ctx *c = new tc_ctx();
  Sizes &s = c->sz;
  s.Nr = Nr;
  s.Nt = Ntheta;
  s.Nz = Nz;
  s.M = (Ntheta - 1) / 3;
  s.K = (Nz - 1) / 3;
  s.NM = s.M + 1;
  s.NK = 2 * s.K + 1;
  s.nmode = s.NM * s.NK;
  c->has_T = (Ra != 0.0);
  s.nf = c->has_T ? 4 : 3;
  s.S = (long long)Nr * s.nmode;
  c->eta = eta;
  c->Lz = Lz;
  c->Re_i = Re_i;
  c->Re_o = Re_o;
  c->Ra = Ra;
  c->Pr = Pr;
  c->Gr = c->has_T ? Ra / Pr : 0.0;
  c->r_i = eta / (1.0 - eta);
  c->r_o = 1.0 / (1.0 - eta);
  try {
    build_tables(c);
    build_base(c);
    allocate(c);
    upload_tables(c);
    setup_nonlinear(c);
    setup_linear(c);
    alignas(64) unsigned char vmap[128];
    // the DFT matrix's slices for the tensor-core transforms (and a TMA
    // tensor map of V that the driver accepts)
    if (theta_tc_supported(s) && theta_tc_map(vmap, c->V, s)) {
      std::vector<unsigned short> tab;
      build_theta_dft(s.Nt, s.M, tab);
      c->d_dft_tc = dalloc<unsigned char>(c, theta_tc_table_bytes());
      ck(cudaMemcpy(c->d_dft_tc, tab.data(), theta_tc_table_bytes(), cudaMemcpyHostToDevice));
      setup_theta_tc();
    }
    if (zinv_tc_supported(s)) {
      std::vector<unsigned short> tab;
      build_zinv_dft(s.Nz, s.K, tab);
      c->d_dft_ztc = dalloc<unsigned char>(c, zinv_tc_table_bytes());
      ck(cudaMemcpy(c->d_dft_ztc, tab.data(), zinv_tc_table_bytes(), cudaMemcpyHostToDevice));
      setup_zinv_tc();
    }
    if (c->smem_zinv > 227 * 1024 || c->smem_theta > 227 * 1024 || c->smem_zfwd > 227 * 1024 ||
        c->smem32_zinv > 227 * 1024 || c->smem32_theta > 227 * 1024 ||
        c->smem32_zfwd > 227 * 1024) {
      tc_destroy(c);
      return TC_ERR_UNSUPPORTED;
    }
    ck(cudaMemcpy(c->X, c->base_dev, c->base.size() * sizeof(double), cudaMemcpyDeviceToDevice));
    launch_factor_poisson(c);
    ck(cudaGetLastError());
    ck(cudaDeviceSynchronize());
  } catch (const std::bad_alloc &) {
    tc_destroy(c);
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    std::fprintf(stderr, "libtc: CUDA error %s\n", cudaGetErrorString(e.e));
    tc_destroy(c);
    return TC_ERR_CUDA;
  }
  *out = c;
  return TC_OK;
}

tc_status tc_destroy(tc_ctx *c) {
  if (!c) return TC_OK;
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_graph) cudaGraphDestroy(c->step_graph);
  for (tc_ctx::CachedGraph *cg : {&c->rec_graph, &c->adj_graph}) {
    if (cg->exec) cudaGraphExecDestroy(cg->exec);
    if (cg->g) cudaGraphDestroy(cg->g);
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (void *p : c->allocs) cudaFree(p);
  if (c->h_step) cudaFreeHost(c->h_step);
  for (auto &t : c->timers)
    for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
  delete c;
  return TC_OK;
}

tc_status tc_set_option(tc_ctx *c, const char *key, double v) {
  if (!c || !key) return TC_ERR_ARG;
  const std::string k(key);
  if (!std::isfinite(v)) return TC_ERR_ARG;
  ++c->gen;   // any option may change a launch parameter of the step
  if (k == "cfl") {
    if (!(v > 0.0)) return TC_ERR_ARG;
    c->cfl = v;
  } else if (k == "dt_max") {
    if (!(v > 0.0)) return TC_ERR_ARG;
    c->dt_max = v;
  } else if (k == "cfl_limit") {
    if (v < 0.0) return TC_ERR_ARG;
    c->cfl_limit = v;
  } else if (k == "check") {
    c->check = v != 0.0;
  } else if (k == "tile_mb" || k == "tile_lb" || k == "tile_mbf") {
    if (v < 0.0 || v > 64.0 || v != (double)(int)v) return TC_ERR_ARG;
    const int old_mb = c->tile_mb, old_lb = c->tile_lb, old_mbf = c->tile_mbf;
    if (k == "tile_mb") c->tile_mb = (int)v;
    else if (k == "tile_lb") c->tile_lb = (int)v;
    else c->tile_mbf = (int)v;
    setup_nonlinear(c);
    const bool fits = (c->precision == 1)
        ? (c->smem32_zinv <= 227 * 1024 && c->smem32_theta <= 227 * 1024 && c->smem32_zfwd <= 227 * 1024)
        : (c->smem_zinv <= 227 * 1024 && c->smem_theta <= 227 * 1024 && c->smem_zfwd <= 227 * 1024);
    if (!fits) {
      c->tile_mb = old_mb;
      c->tile_lb = old_lb;
      c->tile_mbf = old_mbf;
      setup_nonlinear(c);
      return TC_ERR_UNSUPPORTED;
    }
  } else if (k == "tile_mb_adj") {
    if (v < 0.0 || v > 8.0 || v != (double)(int)v) return TC_ERR_ARG;
    c->tile_mb_adj = (int)v;
  } else if (k == "precision") {
    if (v != 0.0 && v != 1.0) return TC_ERR_ARG;
    if (v == 1.0 && c->eps_c != 0.0) return TC_ERR_UNSUPPORTED;
    if (v == 1.0 && !c->X32) {
      try {
        c->X32 = dalloc<float2>(c, (size_t)c->sz.nf * c->sz.S);
      } catch (const std::bad_alloc &) {
        return TC_ERR_OOM;
      }
    }
    c->precision = (int)v;
  } else if (k == "n_corr") {
    if (v < 1.0 || v > 16.0 || v != (double)(int)v) return TC_ERR_ARG;
    c->n_corr = (int)v;
  } else if (k == "flux_constraint") {
    if (v != 0.0 && v != 1.0) return TC_ERR_ARG;
    if ((int)v == c->flux) return TC_OK;
    if (!c->flux_ug) {
      try {
        c->flux_ug = dalloc<double>(c, c->sz.Nr);
      } catch (const std::bad_alloc &) {
        return TC_ERR_OOM;
      }
    }
    try {
      c->flux = (int)v;
      c->lin.flux_ug = c->flux ? c->flux_ug : nullptr;
      build_base(c);
      ck(cudaMemcpyAsync(c->base_dev, c->base.data(), c->base.size() * sizeof(double),
                         cudaMemcpyHostToDevice, c->stream));
      // refactor at the next step, which also builds the unit-forcing response
      char *sb = reinterpret_cast<char *>(c->scal);
      ck(cudaMemsetAsync(sb + offsetof(DevScalars, dt_factored), 0, sizeof(double), c->stream));
      ck(cudaStreamSynchronize(c->stream));
    } catch (const CudaError &e) {
      return fail_cuda(c, e.e);
    }
  } else if (k == "eps_centrifugal") {
    if (!c->has_T || (v != 0.0 && c->precision == 1)) return TC_ERR_UNSUPPORTED;
    c->eps_c = v;
    c->nl.eps_c = v;
  } else if (k == "memory_budget") {
    if (v < 0.0 || v != std::floor(v) || v > 9.0e15) return TC_ERR_ARG;
    c->mem_budget = (size_t)v;
  } else if (k == "tensor_theta") {
    if (v != 0.0 && v != 1.0) return TC_ERR_ARG;
    c->tensor_theta = (int)v;
  } else if (k == "tensor_z") {
    if (v != 0.0 && v != 1.0) return TC_ERR_ARG;
    c->tensor_z = (int)v;
  } else if (k == "selftest_no_copy") {
    c->selftest_no_copy = v != 0.0;
  } else if (k == "timing") {
    c->timing = v != 0.0;
  } else if (k == "graph") {
    c->use_graph = v != 0.0;
  } else {
    return TC_ERR_ARG;
  }
  return TC_OK;
}

tc_status tc_set_stream(tc_ctx *c, void *stream) {
  if (!c) return TC_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return TC_OK;
}

tc_status tc_get_info(const tc_ctx *c, tc_info *o) {
  if (!c || !o) return TC_ERR_ARG;
  o->Nr = c->sz.Nr;
  o->Ntheta = c->sz.Nt;
  o->Nz = c->sz.Nz;
  o->M = c->sz.M;
  o->K = c->sz.K;
  o->nfields = c->sz.nf;
  o->coeffs_per_field = c->sz.S;
  o->state_bytes = (long long)c->sz.nf * c->sz.S * 16;
  o->device_bytes = c->device_bytes;
  o->launches = c->launches;
  o->tile_mb = (c->precision == 1) ? c->nl32.MB : c->nl.MB;
  o->tile_lb = (c->precision == 1) ? c->nl32.LB : c->nl.LB;
  o->tile_mbf = (c->precision == 1) ? c->nl32.MBf : c->nl.MBf;
  o->tensor_theta = (c->precision == 0 && c->tensor_theta && c->d_dft_tc) ? 1 : 0;
  o->tensor_z = (c->precision == 0 && c->tensor_z && c->d_dft_ztc) ? 1 : 0;
  return TC_OK;
}

tc_status tc_set_state(tc_ctx *c, const void *spec, int where) {
  if (!c || !spec || (where != 0 && where != 1)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const size_t bytes = (size_t)16 * c->sz.nf * c->sz.S;
  try {
    // stage in Xp, check on the device, commit only a valid state
    ck(cudaMemcpyAsync(c->Xp, spec, bytes,
                       where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return commit_staged_state(c);
}
tc_status tc_get_state(const tc_ctx *c, void *spec, int where) {
  if (!c || !spec || (where != 0 && where != 1)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const size_t bytes = (size_t)16 * c->sz.nf * c->sz.S;
  // the copy is ordered after the work queued on the stream; one wait
  cudaError_t e = cudaMemcpyAsync(spec, c->X, bytes,
                                  where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail_cuda(const_cast<tc_ctx *>(c), e);
  return TC_OK;
}

tc_status tc_get_pressure(const tc_ctx *c, void *spec, int where) {
  if (!c || !spec || (where != 0 && where != 1)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  cudaError_t e = cudaMemcpyAsync(spec, c->P, (size_t)16 * c->sz.S,
                                  where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail_cuda(const_cast<tc_ctx *>(c), e);
  return TC_OK;
}

tc_status tc_init_perturbation(tc_ctx *c, const double *psi, int mp, int kp, double amp,
                               const double *tcoef, double amp_T) {
  if (!c || !psi || mp < 0 || kp < 0 || !std::isfinite(amp) || !std::isfinite(amp_T))
    return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const Sizes &s = c->sz;
  if (mp > s.M || kp > s.K) return TC_ERR_ARG;
  const int Nr = s.Nr, NK = s.NK, nk = 2 * kp + 1;
  // psi_c(r, m, k) = (1 - x^2)^2 raw_c(m, k), Hermitian m = 0 column
  std::vector<cplx> ps((size_t)3 * s.S, cplx(0.0, 0.0));
  auto P = [&](int comp, int j, int m, int kk) -> cplx & {
    return ps[(size_t)comp * s.S + (size_t)j * s.nmode + (size_t)m * NK + kk];
  };
  for (int j = 0; j < Nr; ++j) {
    const double x = 2.0 * (c->r[j] - c->r_i) - 1.0;
    const double prof = (1.0 - x * x) * (1.0 - x * x);
    for (int comp = 0; comp < 3; ++comp)
      for (int m = 0; m <= mp; ++m)
        for (int k = -kp; k <= kp; ++k) {
          const double *raw = psi + 2 * (((size_t)comp * (mp + 1) + m) * nk + (k + kp));
          P(comp, j, m, (k + NK) % NK) = prof * cplx(raw[0], raw[1]);
        }
    for (int comp = 0; comp < 3; ++comp) {
      for (int k = 1; k <= s.K; ++k) P(comp, j, 0, NK - k) = std::conj(P(comp, j, 0, k));
      P(comp, j, 0, 0) = cplx(P(comp, j, 0, 0).real(), 0.0);
    }
  }
  // u' = curl psi with the same D1 as the step
  std::vector<double> u((size_t)2 * s.nf * s.S, 0.0);
  const double alpha = 2.0 * M_PI / c->Lz;
  const cplx I(0.0, 1.0);
  for (int j = 1; j < Nr - 1; ++j) {
    const int st = c->s0[j];
    const double r = c->r[j];
    for (int m = 0; m < s.NM; ++m)
      for (int kk = 0; kk < NK; ++kk) {
        const double beta = alpha * (kk <= s.K ? kk : kk - NK);
        cplx d1pz(0, 0), d1rpt(0, 0);
        for (int t = 0; t < kStencil; ++t) {
          d1pz += c->D1[j * kStencil + t] * P(2, st + t, m, kk);
          d1rpt += c->D1[j * kStencil + t] * (c->r[st + t] * P(1, st + t, m, kk));
        }
        const cplx pr = P(0, j, m, kk), pt = P(1, j, m, kk), pz = P(2, j, m, kk);
        const cplx ur = I * (double)m * pz / r - I * beta * pt;
        const cplx ut = I * beta * pr - d1pz;
        const cplx uz = d1rpt / r - I * (double)m * pr / r;
        const size_t o = (size_t)j * s.nmode + (size_t)m * NK + kk;
        u[2 * o] = ur.real();
        u[2 * o + 1] = ur.imag();
        u[2 * (s.S + o)] = ut.real();
        u[2 * (s.S + o) + 1] = ut.imag();
        u[2 * (2 * s.S + o)] = uz.real();
        u[2 * (2 * s.S + o) + 1] = uz.imag();
      }
  }
  const bool withT = c->has_T && tcoef && amp_T != 0.0;
  if (withT) {
    std::vector<cplx> tp((size_t)s.S, cplx(0, 0));
    for (int j = 0; j < Nr; ++j) {
      const double x = 2.0 * (c->r[j] - c->r_i) - 1.0;
      for (int m = 0; m <= mp; ++m)
        for (int k = -kp; k <= kp; ++k) {
          const double *raw = tcoef + 2 * ((size_t)m * nk + (k + kp));
          tp[(size_t)j * s.nmode + (size_t)m * NK + (k + NK) % NK] =
              (1.0 - x * x) * cplx(raw[0], raw[1]);
        }
      for (int k = 1; k <= s.K; ++k)
        tp[(size_t)j * s.nmode + NK - k] = std::conj(tp[(size_t)j * s.nmode + k]);
      tp[(size_t)j * s.nmode] = cplx(tp[(size_t)j * s.nmode].real(), 0.0);
    }
    for (long long i = 0; i < s.S; ++i) {
      u[2 * (3 * s.S + i)] = tp[i].real();
      u[2 * (3 * s.S + i) + 1] = tp[i].imag();
    }
  }
  try {
    // every copy ordered on the context's stream (it may be a non-blocking one)
    ck(cudaMemcpyAsync(c->Xp, u.data(), u.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    unsigned long long zero[2] = {0ull, 0ull};
    ck(cudaMemcpyAsync(c->scal->norm_bits, zero, sizeof(zero), cudaMemcpyHostToDevice,
                       c->stream));
    launch_nonlinear(c, c->Xp, nullptr, nullptr, 1);
    ck(cudaGetLastError());
    unsigned long long nb[2];
    ck(cudaMemcpyAsync(nb, c->scal->norm_bits, sizeof(nb), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    double umax, tmax;
    std::memcpy(&umax, &nb[0], sizeof(double));
    std::memcpy(&tmax, &nb[1], sizeof(double));
    // amp > 0: scale to max|u'| = amp; amp < 0: |amp| is the scale itself
    const double su = (amp < 0.0) ? -amp : ((umax > 0.0) ? amp / umax : 0.0);
    const double sT = !withT ? 0.0 : (amp_T < 0.0) ? -amp_T : ((tmax > 0.0) ? amp_T / tmax : 0.0);
    c->ic_su = su;
    c->ic_sT = sT;
    std::vector<double> X(c->base);
    for (long long i = 0; i < 2 * 3 * s.S; ++i) X[i] += su * u[i];
    if (s.nf == 4)
      for (long long i = 2 * 3 * s.S; i < 2 * 4 * s.S; ++i) X[i] += sT * u[i];
    invalidate_rhs_identity(c);
    ck(cudaMemcpyAsync(c->X, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    DevScalars sc{};
    ck(cudaMemcpyAsync(c->scal, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  c->t = 0.0;
  return TC_OK;
}

tc_status tc_step(tc_ctx *c, int nsteps, double dt, double *dt_used) {
  if (!c || nsteps < 0 || !std::isfinite(dt)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (nsteps == 0) return TC_OK;
  try {
    if (nsteps > c->dt_hist_cap) {
      // device memory added: the difference when the old history is freed,
      // the whole new one when the old one stays (inside the scalars' block)
      const size_t grow = sizeof(double) * (size_t)(c->dt_hist_own ? nsteps - c->dt_hist_cap
                                                                   : nsteps);
      if (over_budget(c, grow)) return TC_ERR_OOM;
      double *h = nullptr;
      if (cudaMalloc(&h, sizeof(double) * nsteps) != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_OOM;
      }
      ck(cudaStreamSynchronize(c->stream));   // the old history may still be in use
      if (c->dt_hist_own) {
        cudaFree(c->dt_hist);
        for (auto &p : c->allocs)
          if (p == c->dt_hist) p = h;
      } else {   // the first history lives in the scalars' allocation
        c->allocs.push_back(h);
      }
      c->dt_hist = h;
      c->dt_hist_own = true;
      c->device_bytes += grow;
      c->dt_hist_cap = nsteps;
      ++c->gen;   // the history pointer is a kernel argument
    }
    char *sb = reinterpret_cast<char *>(c->scal);
    static_assert(offsetof(DevScalars, hist_pos) == offsetof(DevScalars, nonfinite) + sizeof(int),
                  "nonfinite and hist_pos are cleared together");
    ck(cudaMemsetAsync(sb + offsetof(DevScalars, nonfinite), 0, 2 * sizeof(int), c->stream));
    const double dt_fixed = dt > 0.0 ? dt : 0.0;
    if (c->use_graph && !c->timing) {
      const cudaError_t ge = ensure_step_graph(c, dt_fixed);
      if (ge != cudaSuccess) {
        // not capturable here: launch the kernels directly from now on
        cudaGetLastError();
        std::fprintf(stderr, "libtc: step graph unavailable (%s), launching directly\n",
                     cudaGetErrorString(ge));
        c->use_graph = 0;
      }
    }
    if (c->use_graph && !c->timing) {
      for (int n = 0; n < nsteps; ++n) ck(cudaGraphLaunch(c->step_exec, c->stream));
      c->launches += c->graph_launches * nsteps;
    } else {
      for (int n = 0; n < nsteps; ++n) enqueue_step(c, dt_fixed, n);
    }
    ck(cudaGetLastError());
    // the step history and the device scalars, into pinned memory when the
    // history fits (asynchronous copies, one wait)
    std::vector<double> hist_big;
    DevScalars sc_big;
    const bool pinned = nsteps <= tc_ctx::kPinnedHist;
    if (!pinned) hist_big.resize(nsteps);
    double *hist = pinned ? reinterpret_cast<double *>(c->h_step + tc_ctx::kPinnedScal)
                          : hist_big.data();
    DevScalars *scp = pinned ? reinterpret_cast<DevScalars *>(c->h_step) : &sc_big;
    if (pinned && !c->dt_hist_own) {   // scalars and history in one copy
      ck(cudaMemcpyAsync(c->h_step, c->scal, tc_ctx::kPinnedScal + sizeof(double) * nsteps,
                         cudaMemcpyDeviceToHost, c->stream));
    } else {
      ck(cudaMemcpyAsync(hist, c->dt_hist, sizeof(double) * nsteps, cudaMemcpyDeviceToHost,
                         c->stream));
      ck(cudaMemcpyAsync(scp, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    }
    ck(cudaStreamSynchronize(c->stream));
    const DevScalars sc = *scp;
    for (int n = 0; n < nsteps; ++n) c->t += hist[n];
    if (dt_used) std::memcpy(dt_used, hist, sizeof(double) * nsteps);
    if (sc.timeout) return TC_ERR_TIMEOUT;
    if (c->check && sc.nonfinite) return TC_ERR_NONFINITE;
    if (c->cfl_limit > 0.0 && sc.rate_last * sc.dt > c->cfl_limit) return TC_ERR_CFL;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_get_clock(const tc_ctx *c, double *t, double *dt_prev) {
  if (!c) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (dt_prev) {
    // the device value: tc_stage_solve and the adjoint entry points also run
    // the step policy
    double v = 0.0;
    cudaError_t e = cudaMemcpyAsync(&v, &c->scal->dt_prev, sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(const_cast<tc_ctx *>(c), e);
    *dt_prev = v;
  }
  if (t) *t = c->t;
  return TC_OK;
}

tc_status tc_set_clock(tc_ctx *c, double t, double dt_prev) {
  if (!c || !std::isfinite(t) || !std::isfinite(dt_prev) || dt_prev < 0.0) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  try {
    // a pageable source: the copy is staged before the call returns
    ck(cudaMemcpyAsync(&c->scal->dt_prev, &dt_prev, sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  c->t = t;
  return TC_OK;
}

tc_status tc_nonlinear(tc_ctx *c, const void *state_dev, void *n_dev, double *cfl_rate) {
  if (!c || !state_dev || !n_dev) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  try {
    unsigned long long *rb = &c->scal->rate_bits;
    unsigned long long z = 0ull;
    int zero = 0, to = 0;
    ck(cudaMemcpyAsync(rb, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream));
    ck(cudaMemcpyAsync(&c->scal->timeout, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    launch_nonlinear(c, static_cast<const double2 *>(state_dev), static_cast<double2 *>(n_dev), rb,
                     0);
    ck(cudaGetLastError());
    unsigned long long bits;
    ck(cudaMemcpyAsync(&bits, rb, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaMemcpyAsync(rb, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream));
    ck(cudaMemcpyAsync(&to, &c->scal->timeout, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    if (cfl_rate) std::memcpy(cfl_rate, &bits, sizeof(double));
    if (to) return TC_ERR_TIMEOUT;   // a bounded wait of the tensor-core kernel ran out
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_stage_solve(tc_ctx *c, const void *rhs_dev, double dt, void *x_out_dev,
                         void *p_out_dev) {
  if (!c || !rhs_dev || !x_out_dev || !(dt > 0.0) || !std::isfinite(dt)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const Sizes &s = c->sz;
  try {
    invalidate_rhs_identity(c);
    ck(cudaMemcpyAsync(c->Yb, rhs_dev, (size_t)16 * s.nf * s.S, cudaMemcpyDeviceToDevice,
                       c->stream));
    ck(cudaMemsetAsync(c->N1, 0, (size_t)16 * s.nf * s.S, c->stream));
    launch_dt_policy(c, dt, -1);
    launch_refactor(c);
    launch_stage(c, c->N1, static_cast<double2 *>(x_out_dev), c->P);
    if (p_out_dev)
      ck(cudaMemcpyAsync(p_out_dev, c->P, (size_t)16 * s.S, cudaMemcpyDeviceToDevice, c->stream));
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(c->stream));
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_diagnostics(tc_ctx *c, tc_diag *o) {
  if (!c || !o) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  try {
    launch_diagnostics(c);
    ck(cudaGetLastError());
    double h[13];
    ck(cudaMemcpyAsync(h, c->diag_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    unsigned long long cb = 0ull;
    ck(cudaMemcpyAsync(&cb, &c->scal->corr_bits, sizeof(cb), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    std::memcpy(&o->corr_diff, &cb, sizeof(double));
    o->t = c->t;
    o->dt = h[0];
    o->E = h[1];
    o->E_pert = h[2];
    o->torque_i = h[3];
    o->torque_o = h[4];
    o->P_wall = h[5];
    o->eps = h[6];
    o->buoy_work = h[7];
    o->Nu_i = h[8];
    o->Nu_o = h[9];
    o->div_max = h[10];
    o->div_rms = h[11];
    o->cfl = h[12];
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

}  // extern "C"

namespace tc {
namespace {

void ensure_adjoint(tc_ctx *c) {
  if (c->Phys) return;
  const Sizes &s = c->sz;
  // all or nothing: the buffers count as present once the last one exists
  const size_t need = 16 * ((size_t)3 * s.nf * s.Nr * s.Nz * s.NM + (size_t)5 * s.nf * s.S +
                            (size_t)s.Nr * s.Nz * 2 * s.nf * s.Nt);
  if (over_budget(c, need)) throw std::bad_alloc();
  c->Va = dalloc<double2>(c, (size_t)3 * s.nf * s.Nr * s.Nz * s.NM);
  c->Gdr = dalloc<double2>(c, (size_t)s.nf * s.S);
  c->Rb = dalloc<double2>(c, (size_t)s.nf * s.S);
  c->Ybar = dalloc<double2>(c, (size_t)s.nf * s.S);
  c->Nb = dalloc<double2>(c, (size_t)s.nf * s.S);
  c->Xb = dalloc<double2>(c, (size_t)s.nf * s.S);
  c->Phys = dalloc<double2>(c, (size_t)s.Nr * s.Nz * 2 * s.nf * s.Nt);
  setup_nonlinear_adjoint(c);
}

}  // namespace
}  // namespace tc

extern "C" {

namespace {

// Reverse sweep of one step given its linearisation points: X^n, the
// predictor state X* and the physical-grid fields of X^n and (nullable) of X*.
// lam: lambda^(n+1) in, lambda^n out.  The factors and influence data must be
// those of dt.
void enqueue_adjoint_sweep(tc_ctx *c, const double2 *Xn, const double2 *Xs,
                           const double2 *phys, const double2 *phys_s, double2 *lam) {
  launch_stage_adjoint(c, lam, c->Rb);                      // corrector stage
  launch_stage_split_adjoint(c, c->Rb, c->Ybar, c->Nb, 0);
  launch_nonlinear_adjoint(c, Xs, c->Nb, c->Xb, 0, phys_s); // N(X*)
  launch_stage_adjoint(c, c->Xb, c->Rb);                    // predictor stage
  launch_stage_split_adjoint(c, c->Rb, c->Ybar, c->Nb, 1);
  launch_rhs_adjoint(c, c->Ybar, lam, c->Nb);
  launch_nonlinear_adjoint(c, Xn, c->Nb, lam, 1, phys);     // N(X^n)
  launch_herm_project(c, lam);
}

tc_status adjoint_supported(const tc_ctx *c) {
  // the adjoint is of the default scheme: FP64, one corrector, no flux
  // constraint, no centrifugal buoyancy
  if (c->precision != 0 || c->n_corr != 1 || c->flux || c->eps_c != 0.0)
    return TC_ERR_UNSUPPORTED;
  return TC_OK;
}

// Record of one step: X^n, X* (nf S complex each), then the physical fields
// of X^n and of X* (Nr Nz 2 nf Nt complex each).
long long phys_doubles2(const tc_ctx *c) {
  const Sizes &s = c->sz;
  return (long long)s.Nr * s.Nz * 2 * s.nf * s.Nt;
}
long long record_doubles2(const tc_ctx *c) {
  return 2LL * c->sz.nf * c->sz.S + 2 * phys_doubles2(c);
}

}  // namespace

tc_status tc_adjoint_step(tc_ctx *c, const void *state_n_dev, double dt, void *adj_dev) {
  if (!c || !state_n_dev || !adj_dev || !(dt > 0.0) || !std::isfinite(dt)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (adjoint_supported(c) != TC_OK) return TC_ERR_UNSUPPORTED;
  const double2 *Xn = static_cast<const double2 *>(state_n_dev);
  double2 *lam = static_cast<double2 *>(adj_dev);
  try {
    ensure_adjoint(c);
    invalidate_rhs_identity(c);
    int zero = 0;
    ck(cudaMemcpyAsync(&c->scal->timeout, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    // forward internals of the step at X^n: only the predictor state X* is
    // needed (the linearisation point of N(X*)); N(X*) itself is not, since
    // the corrector stage is linear in its right-hand side and the adjoint
    // of the nonlinear stage recomputes its own transforms of X*
    launch_nonlinear(c, Xn, c->N0, nullptr, 0, c->Phys);   // keeps the physical fields of X^n
    launch_dt_policy(c, dt, -1);
    launch_refactor(c);
    launch_rhs(c, Xn, c->N0);
    launch_stage(c, c->N0, c->Xp, c->P);
    enqueue_adjoint_sweep(c, Xn, c->Xp, c->Phys, nullptr, lam);
    ck(cudaGetLastError());
    int to = 0;
    ck(cudaMemcpyAsync(&to, &c->scal->timeout, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    if (to) return TC_ERR_TIMEOUT;
  } catch (const std::bad_alloc &) {
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}


tc_status tc_record_bytes_per_step(const tc_ctx *c, long long *bytes) {
  if (!c || !bytes) return TC_ERR_ARG;
  *bytes = 16 * record_doubles2(c);
  return TC_OK;
}

tc_status tc_step_record(tc_ctx *c, int nsteps, double dt, void *record_dev,
                         long long record_bytes) {
  if (!c || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return TC_ERR_ARG;
  if (nsteps > 0 && (!record_dev || record_bytes < 16 * record_doubles2(c) * nsteps))
    return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (adjoint_supported(c) != TC_OK) return TC_ERR_UNSUPPORTED;
  if (nsteps == 0) return TC_OK;
  const Sizes &s = c->sz;
  const long long S = s.S;
  try {
    ensure_adjoint(c);
    char *sb = reinterpret_cast<char *>(c->scal);
    ck(cudaMemsetAsync(sb + offsetof(DevScalars, nonfinite), 0, sizeof(int), c->stream));
    double2 *rec = static_cast<double2 *>(record_dev);
    run_cached(c, c->rec_graph, record_dev, nullptr, nsteps, dt, [&]() {
    for (int n = 0; n < nsteps; ++n) {
      double2 *rX = rec + (long long)n * record_doubles2(c);
      double2 *rXs = rX + (long long)s.nf * S;
      double2 *rP = rXs + (long long)s.nf * S;
      double2 *rPs = rP + phys_doubles2(c);
      cudaMemcpyAsync(rX, c->X, 16 * (size_t)s.nf * S, cudaMemcpyDeviceToDevice, c->stream);
      // one step (the default scheme: one corrector), its predictor state and
      // both nonlinear evaluations' physical fields written straight into
      // the record
      launch_nonlinear(c, c->X, c->N0, &c->scal->rate_bits, 0, rP);
      launch_dt_policy(c, dt, -1);
      launch_refactor(c);
      launch_rhs(c, c->X, c->N0);
      launch_stage(c, c->N0, rXs, c->P);
      launch_nonlinear(c, rXs, c->N1, nullptr, 0, rPs);
      launch_stage(c, c->N1, c->X, c->P, rXs);
    }
    });
    ck(cudaGetLastError());
    DevScalars sc;
    ck(cudaMemcpyAsync(&sc, c->scal, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    c->t += dt * nsteps;
    if (sc.timeout) return TC_ERR_TIMEOUT;
    if (c->check && sc.nonfinite) return TC_ERR_NONFINITE;
  } catch (const std::bad_alloc &) {
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_adjoint_steps(tc_ctx *c, int nsteps, const void *record_dev, double dt,
                           void *adj_dev) {
  if (!c || nsteps < 0 || !adj_dev || !(dt > 0.0) || !std::isfinite(dt)) return TC_ERR_ARG;
  if (nsteps > 0 && !record_dev) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (adjoint_supported(c) != TC_OK) return TC_ERR_UNSUPPORTED;
  if (nsteps == 0) return TC_OK;
  const Sizes &s = c->sz;
  const double2 *rec = static_cast<const double2 *>(record_dev);
  double2 *lam = static_cast<double2 *>(adj_dev);
  try {
    ensure_adjoint(c);
    invalidate_rhs_identity(c);
    int zero = 0;
    ck(cudaMemcpyAsync(&c->scal->timeout, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    run_cached(c, c->adj_graph, record_dev, adj_dev, nsteps, dt, [&]() {
      launch_dt_policy(c, dt, -1);   // the factors of dt
      launch_refactor(c);
      for (int n = nsteps - 1; n >= 0; --n) {
        const double2 *rX = rec + (long long)n * record_doubles2(c);
        const double2 *rXs = rX + (long long)s.nf * s.S;
        const double2 *rP = rXs + (long long)s.nf * s.S;
        enqueue_adjoint_sweep(c, rX, rXs, rP, rP + phys_doubles2(c), lam);
      }
    });
    ck(cudaGetLastError());
    int to = 0;
    ck(cudaMemcpyAsync(&to, &c->scal->timeout, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    if (to) return TC_ERR_TIMEOUT;
  } catch (const std::bad_alloc &) {
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_nonlinear_adjoint(tc_ctx *c, const void *state_dev, const void *nbar_dev,
                               void *xbar_dev) {
  if (!c || !state_dev || !nbar_dev || !xbar_dev) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (c->eps_c != 0.0) return TC_ERR_UNSUPPORTED;
  try {
    ensure_adjoint(c);
    launch_nonlinear_adjoint(c, static_cast<const double2 *>(state_dev),
                             static_cast<const double2 *>(nbar_dev),
                             static_cast<double2 *>(xbar_dev), 0);
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(c->stream));
  } catch (const std::bad_alloc &) {
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_stage_solve_adjoint(tc_ctx *c, const void *xbar_dev, double dt, void *rbar_dev) {
  if (!c || !xbar_dev || !rbar_dev || !(dt > 0.0) || !std::isfinite(dt)) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  if (c->flux) return TC_ERR_UNSUPPORTED;
  try {
    ensure_adjoint(c);
    invalidate_rhs_identity(c);
    int zero = 0;
    ck(cudaMemcpyAsync(&c->scal->timeout, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    launch_dt_policy(c, dt, -1);
    launch_refactor(c);
    launch_stage_adjoint(c, static_cast<const double2 *>(xbar_dev), static_cast<double2 *>(rbar_dev));
    ck(cudaGetLastError());
    int to = 0;
    ck(cudaMemcpyAsync(&to, &c->scal->timeout, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    if (to) return TC_ERR_TIMEOUT;
  } catch (const std::bad_alloc &) {
    return TC_ERR_OOM;
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  return TC_OK;
}

tc_status tc_objective(tc_ctx *c, double *J, void *grad_dev) {
  if (!c || !J) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  tc_diag d;
  tc_status st = tc_diagnostics(c, &d);
  if (st != TC_OK) return st;
  *J = d.E_pert;
  if (grad_dev) {
    try {
      launch_objective_grad(c, c->X, static_cast<double2 *>(grad_dev));
      ck(cudaGetLastError());
      ck(cudaStreamSynchronize(c->stream));
    } catch (const CudaError &e) {
      return fail_cuda(c, e.e);
    }
  }
  return TC_OK;
}

tc_status tc_init_perturbation_adjoint(tc_ctx *c, const void *lam_dev, int mp, int kp,
                                       double *psi_bar, double *tcoef_bar) {
  if (!c || !lam_dev || !psi_bar || mp < 0 || kp < 0) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  const Sizes &s = c->sz;
  if (mp > s.M || kp > s.K) return TC_ERR_ARG;
  const int Nr = s.Nr, NK = s.NK, nk = 2 * kp + 1;
  std::vector<cplx> lam((size_t)s.nf * s.S);
  try {
    ck(cudaStreamSynchronize(c->stream));
    ck(cudaMemcpyAsync(lam.data(), lam_dev, sizeof(cplx) * lam.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    ck(cudaStreamSynchronize(c->stream));
  } catch (const CudaError &e) {
    return fail_cuda(c, e.e);
  }
  auto L = [&](int f, int j, int m, int kk) -> cplx {
    return lam[(size_t)f * s.S + (size_t)j * s.nmode + (size_t)m * NK + kk];
  };
  // transpose of u' = s_u Zw curl(psi): psi_bar per component (interior rows)
  std::vector<cplx> pb((size_t)3 * s.S, cplx(0.0, 0.0));
  auto PB = [&](int comp, int j, int m, int kk) -> cplx & {
    return pb[(size_t)comp * s.S + (size_t)j * s.nmode + (size_t)m * NK + kk];
  };
  const double alpha = 2.0 * M_PI / c->Lz;
  const cplx I(0.0, 1.0);
  const double su = c->ic_su;
  for (int j = 1; j < Nr - 1; ++j) {
    const int st = c->s0[j];
    const double r = c->r[j];
    for (int m = 0; m < s.NM; ++m)
      for (int kk = 0; kk < NK; ++kk) {
        const double beta = alpha * (kk <= s.K ? kk : kk - NK);
        const cplx ur = su * L(0, j, m, kk), ut = su * L(1, j, m, kk), uz = su * L(2, j, m, kk);
        // u_r = (i m / r) psi_z - i beta psi_theta
        PB(2, j, m, kk) += std::conj(I * (double)m / r) * ur;
        PB(1, j, m, kk) += std::conj(-I * beta) * ur;
        // u_theta = i beta psi_r - D1 psi_z
        PB(0, j, m, kk) += std::conj(I * beta) * ut;
        // u_z = (1/r) D1(r psi_theta) - (i m / r) psi_r
        PB(0, j, m, kk) += std::conj(-I * (double)m / r) * uz;
        for (int t = 0; t < kStencil; ++t) {
          PB(2, st + t, m, kk) -= c->D1[j * kStencil + t] * ut;
          PB(1, st + t, m, kk) += (c->D1[j * kStencil + t] * c->r[st + t] / r) * uz;
        }
      }
  }
  // transpose of the Hermitian fix and of the radial profile
  for (int comp = 0; comp < 3; ++comp)
    for (int m = 0; m <= mp; ++m)
      for (int k = -kp; k <= kp; ++k) {
        cplx acc(0.0, 0.0);
        for (int j = 0; j < Nr; ++j) {
          const double x = 2.0 * (c->r[j] - c->r_i) - 1.0;
          const double prof = (1.0 - x * x) * (1.0 - x * x);
          cplx v;
          if (m == 0 && k < 0) {
            v = 0.0;        // overwritten by the fix: no influence
          } else if (m == 0 && k > 0) {
            v = PB(comp, j, 0, k) + std::conj(PB(comp, j, 0, NK - k));
          } else if (m == 0 && k == 0) {
            v = cplx(PB(comp, j, 0, 0).real(), 0.0);
          } else {
            v = PB(comp, j, m, (k + NK) % NK);
          }
          acc += prof * v;
        }
        double *o = psi_bar + 2 * (((size_t)comp * (mp + 1) + m) * nk + (k + kp));
        o[0] = acc.real();
        o[1] = acc.imag();
      }
  if (tcoef_bar) {
    for (int m = 0; m <= mp; ++m)
      for (int k = -kp; k <= kp; ++k) {
        cplx acc(0.0, 0.0);
        if (s.nf == 4 && c->ic_sT != 0.0) {
          for (int j = 0; j < Nr; ++j) {
            const double x = 2.0 * (c->r[j] - c->r_i) - 1.0;
            cplx v;
            if (m == 0 && k < 0)
              v = 0.0;
            else if (m == 0 && k > 0)
              v = L(3, j, 0, k) + std::conj(L(3, j, 0, NK - k));
            else if (m == 0 && k == 0)
              v = cplx(L(3, j, 0, 0).real(), 0.0);
            else
              v = L(3, j, m, (k + NK) % NK);
            acc += (1.0 - x * x) * c->ic_sT * v;
          }
        }
        double *o = tcoef_bar + 2 * ((size_t)m * nk + (k + kp));
        o[0] = acc.real();
        o[1] = acc.imag();
      }
  }
  return TC_OK;
}

tc_status tc_get_ic_scales(const tc_ctx *c, double *s_u, double *s_T) {
  if (!c || !s_u || !s_T) return TC_ERR_ARG;
  *s_u = c->ic_su;
  *s_T = c->ic_sT;
  return TC_OK;
}

tc_status tc_debug_flags(unsigned *flags, int clear) {
  if (!flags) return TC_ERR_ARG;
  *flags = 0;
#ifndef TC_DEBUG
  (void)clear;
  return TC_ERR_UNSUPPORTED;
#else
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_CUDA;
  }
  *flags = debug_word_nonlinear(clear) | debug_word_linear(clear);
  return TC_OK;
#endif
}

tc_status tc_get_timing(tc_ctx *c, tc_kernel_time *out, int cap, int *count) {
  if (!c || (!out && cap > 0) || !count) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail_cuda(c, e);
  int n = 0;
  for (int k = 0; k < KNUM; ++k) {
    KernelTimer &t = c->timers[k];
    if (t.used == 0) continue;
    double ms = 0.0;
    for (int i = 0; i < t.used; ++i) {
      float f = 0.0f;
      e = cudaEventElapsedTime(&f, t.ev[2 * i], t.ev[2 * i + 1]);
      if (e != cudaSuccess) return fail_cuda(c, e);
      ms += f;
    }
    if (n < cap) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
      out[n].launches = t.used;
      out[n].ms = ms;
    }
    ++n;
  }
  *count = n;
  return TC_OK;
}

tc_status tc_reset_timing(tc_ctx *c) {
  if (!c) return TC_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail_cuda(c, e);
  for (auto &t : c->timers) t.used = 0;
  return TC_OK;
}

}  // extern "C"
