// Internal declarations of libtc: context, device tables and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "tc.h"

namespace tc {

// Index checks of the debug build (compiled with -DTC_DEBUG; libtc_debug.so).
// dbg_in(i, n, site) is true when 0 <= i < n.  In the debug build an index
// out of that range sets bit `site` of a device word of this translation unit
// and returns false, and the caller skips the access: a bad index is
// recorded, never dereferenced, and never traps.  tc_debug_flags reads the
// words.  In the normal build dbg_in is the constant true and the checks
// compile away.
enum DbgSite {
  DBG_ZINV_X, DBG_ZINV_V, DBG_THETA_V, DBG_THETA_W, DBG_THETA_PHYS, DBG_ZFWD_W, DBG_ZFWD_N,
  DBG_FFT_SMEM, DBG_RHS, DBG_PRHS, DBG_HRHS, DBG_SWEEP_X, DBG_SWEEP_COPY, DBG_ALPHA,
  DBG_CORRECT, DBG_NSITES
};
#ifdef TC_DEBUG
static __device__ unsigned int g_dbg_word;
__device__ __forceinline__ bool dbg_in(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  atomicOr(&g_dbg_word, 1u << site);
  return false;
}
#else
__device__ __forceinline__ constexpr bool dbg_in(long long, long long, int) { return true; }
#endif
// Host side: this translation unit's word (0 in the normal build); clear != 0
// resets it.  One reader per .cu file that checks indices.
unsigned debug_word_nonlinear(int clear);
unsigned debug_word_linear(int clear);

constexpr int kStencil = 9;   // radial FD stencil (Sec. 2.1: 9 points by default)
constexpr int kBand = 8;      // half bandwidth of the radial operators
constexpr int kBandW = 17;    // stored band entries per row (8 lower, diag, 8 upper)
constexpr double kCN = 0.5;   // implicit weight of the predictor-corrector
constexpr int kSweepRows = 16;    // rows per staged chunk of band factors
constexpr int kSweepOps = 16;     // operators (|k| values) per sweep CTA
constexpr int kSweepStages = 3;   // depth of the shared-memory ring

// Division by a divisor fixed at set-up: q = (t + ((n - t) >> s1)) >> s2 with
// t = umulhi(m, n) (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994), exact for every 32-bit n.
struct FastDiv {
  unsigned m;
  int s1, s2;
};

struct FFTPlan {
  int n;
  int npass;
  int radix[16];
  // twiddles of pass p (Ns > 1), w = exp(-2 pi i / (Ns R)), slot i of k at
  // tw_off[p] + i Ns + k: radix 2, 3, 5 w^(q k) in slot q - 1; radix 4 and 8
  // cosine-tangent forms of w^k, w^2k (and w^4k, w^k e^(-i pi/4), its square);
  // (R - 1) Ns slots reserved per pass, n - 1 in all
  int tw_off[16];
  FastDiv div_nb[16];   // division by n / radix[p]
  FastDiv div_ns[16];   // division by Ns of pass p
};

FastDiv make_fastdiv(unsigned d);
FFTPlan make_plan(int n);
// Pass-major twiddle table of a plan: n entries (the last one unused).
void fill_plan_twiddles(const FFTPlan &pl, double2 *out);

// Host helpers shared by the set-up code (tc_host.cu).
void fd_weights(double x0, const double *x, int n, double w[3][kStencil]);

// Axial wavenumber index k of stored index kk (FFT order: 0..K, then -K..-1).
__host__ __device__ __forceinline__ int kval(int kk, int K, int NK) {
  return kk <= K ? kk : kk - NK;
}

// Problem sizes.
struct Sizes {
  int Nr, Nt, Nz, M, K, NM, NK, nmode, nf;
  long long S;  // Nr * nmode coefficients per field (< 2^31: Nr <= 1024, Nt, Nz <= 1024)
};

// Device-side radial tables (device pointers).
struct Radial {
  const double *r, *inv_r, *D1, *D2, *dr_min, *wr;  // wr = quadrature w_j r_j
  const int *s0;                                     // stencil start per node
  const double *Lw;   // [Nr][9] D2 + D1/r_j: the radial part of L in one stencil
  const double *Dw;   // [Nr][9] (1/r_j) D1 r_s: the radial part of div
  // transposed stencils: [Nr][kTrans] the rows j whose stencil holds node n,
  // ascending, -1 after the last.  At most 13 for Nr >= 18 (the 5 rows whose
  // stencil is clamped to a wall plus 8 centred ones); with Nr <= 17 every row
  // can hold node n, so at most 17.
  const int *tj;
};
constexpr int kTrans = 20;

// Scalars shared between kernels on the device.
struct DevScalars {
  double dt;            // step in use
  double dt_factored;   // step the Helmholtz factors belong to
  double dt_prev;       // previous step (dynamic policy)
  unsigned long long rate_bits;   // CFL rate of the last start-of-step state
  unsigned long long norm_bits[2];  // max |u'|, max |T'| (initial condition)
  unsigned long long chk_bits[2];   // tc_set_state: max |x|, max Hermitian defect
  double rate_last;     // rate read by the policy
  int refactor;         // 1 when the factors must be rebuilt this step
  int nonfinite;        // set when a solve produced NaN/Inf
  int hist_pos;         // next slot of the step history of the current tc_step call
                        // (next to nonfinite: tc_step clears both with one memset)
  int timeout;          // set when a bounded device-side wait gave up
  unsigned long long corr_bits;   // max |X_corr - X_prev| of the last corrector
  // 1 while X, Yb, N1 and P are the last corrector's state, right-hand side,
  // nonlinear term and pressure (k_correct sets it; every entry point that
  // changes one of them outside a step clears it): k_rhs may then take L X
  // from that stage's equation instead of the stencil
  int rhs_ident;
  double dt_old;        // step of the stage that produced the current state
  double idt, idt_old;  // 1/dt and 1/dt_old, set with them by the step policy
};

// Parameters of the nonlinear stage.
struct NLParams {
  Sizes sz;
  Radial rad;
  double alpha;         // 2 pi / Lz
  double Gr;            // Ra / Pr
  double dth, dz;       // grid spacings in theta and z
  // CFL rate without divisions on the device: [r][2] = 1/dr_min(r),
  // 1/(r dth), and 1/dz (the one thread per CTA that scales the CTA's maxima
  // would otherwise run three FP64 divisions, each a chain of FP64
  // instructions that costs the whole warp's turns)
  const double *cfl_inv;
  double inv_dz;
  const double *betak;  // alpha k per stored axial index (FP64)
  double zscale;        // 1/(2 Ntheta Nz): forward scale with the 1/2 of k_theta's unpacking
  int MB;               // m columns per CTA in k_zinv (and the adjoint z kernels)
  int MBf;              // m columns per CTA in k_zfwd
  int LB;               // z rows per CTA in the theta kernel
  FFTPlan pz, pt;
  const double2 *twz, *twt;   // pass-major twiddle tables of pz, pt (FP64 master copy)
  // mixed precision: the transforms carry only the perturbation u' = u - U(r)
  // (FP32); the products with the mean mode U are added in FP64 in k_zfwd
  int mixed;
  const double2 *Xfull;       // state (mixed only)
  const double *prof;         // [r][8]: U_theta, U_z, dU_theta/dr, dU_z/dr, dTbar/dr, T mean
  double eps_c;               // centrifugal buoyancy: advection weighted by 1 - eps_c T (FP64 only)
  // fixed divisors of the element loops (set_divisors): NK, NM, Nt, Nz, nf,
  // MB and the last m-block's width, MBf and its last block's width
  FastDiv fNK, fNM, fNt, fNz, fnf, fMB, fMBl, fMBf, fMBfl;
  // physical-grid fields of the forward transforms, [r][z][2 nf][Nt] complex
  // pairs (value + i d/dtheta, d/dr + i d/dz per component): k_theta writes
  // them when phys_out is set, the adjoint theta kernel reads them instead of
  // transforming the state again when phys_in is set (FP64 only)
  double2 *phys_out;
  const double2 *phys_in;
  // FP32 copies for the mixed form's transform kernels, each entry the FP32
  // rounding of its FP64 counterpart made once on the host: the twiddle
  // tables, the 9-point d/dr weights [r][9], beta = alpha k per stored axial
  // index, 1/r; prof32 [r][2] = U_theta, U_z (written by k_meanprof).  An FP64
  // instruction costs a warp's turn on the FP64 unit (about 64 cycles)
  // however few of its lanes are active, so the FP32 kernels take these
  // values instead of converting per thread.
  const float2 *twz32, *twt32;
  const float *d1_32, *beta32, *inv_r32;
  float *prof32;
};
void set_divisors(NLParams &p);

// Parameters of the linear stage.
struct LinParams {
  Sizes sz;
  Radial rad;
  double alpha;
  double kappaT;        // 1/Pr
  double Re_i, Re_o;
  int nopP, nopH, nopT; // operator counts: Poisson, velocity Helmholtz, T Helmholtz
  int Nrp;              // rows padded to a multiple of kSweepRows
  // band factors, operator-major: L [op][Nrp][8] (sub-diagonals), U [op][Nrp][9]
  // (inverse diagonal, then 8 super-diagonals)
  double *LP, *UP, *LH, *UH, *LT, *UT;
  double *infl;         // influence data [8][Nr][nopP]: pa pb upa uma upb umb za zb
  double *Ainv;         // [4][nopP]
  double *flux_ug;      // axial-flux constraint: (0,0) u_z response to a unit forcing (Nr), or null
  // beta = alpha k per stored axial index (NK) and m as a double (NM), so the
  // per-coefficient kernels convert no integer on the FP64 unit
  const double *betak, *mval;
};

}  // namespace tc

namespace tc {
// Kernels with per-launch timing (option "timing").
enum KernelId {
  KZINV, KTHETA, KZFWD, KDT, KFACTH, KINFL, KRHS, KPRHS, KPOIS, KHRHS, KHELM, KALPHA, KCORR,
  KDIAG, KCHECK, KFLUX, KREGRID, KADJ, KTHETATC, KZINVTC, KNUM
};
extern const char *const kKernelNames[KNUM];

struct KernelTimer {
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  int used = 0;                  // pairs recorded since the last reset
  long long launches = 0;
};
}  // namespace tc

struct tc_ctx {
  tc::Sizes sz;
  double eta, Lz, Re_i, Re_o, Ra, Pr, Gr, r_i, r_o;
  bool has_T;
  double cfl = 0.25, dt_max = 1e-3, cfl_limit = 0.0;
  int check = 1;
  int selftest_no_copy = 0;   // test hook: sweeps never start their copies
  cudaStream_t stream = nullptr;
  bool poisoned = false;
  double t = 0.0;
  // host tables
  std::vector<double> r, D1, D2, w, dr_min;
  std::vector<int> s0;
  std::vector<double> base;     // basic state, interleaved complex [nf][S]
  std::vector<double> Tb_disc;  // discrete conductive profile (Nr)
  // device memory
  std::vector<void *> allocs;
  size_t device_bytes = 0;
  // largest device_bytes allowed for allocations made after tc_create
  // (option "memory_budget"; 0: no limit)
  size_t mem_budget = 0;
  double2 *X, *Xp, *N0, *N1, *Yb, *U0, *P, *V, *W, *alpha_buf, *base_dev;
  double *Ps;   // particular pressure, split planes [2][S]
  double *d_Lw, *d_Dw;
  int *d_tj;
  double *d_r, *d_inv_r, *d_D1, *d_D2, *d_dr, *d_wr;
  int *d_s0;
  double2 *d_twz, *d_twt;
  float *d_f32;          // FP32 tables of NLParams (twiddles, d/dr weights, beta, 1/r)
  float *d_prof32;       // [Nr][2] FP32 mean profiles (mixed form)
  double *d_kmtab;       // LinParams::betak (NK) then mval (NM)
  double *d_cflinv;      // NLParams::cfl_inv (2 Nr)
  // pinned host buffer that tc_step reads the device scalars and the step
  // history into (kPinnedHist steps; longer calls use pageable memory): the
  // copies are then asynchronous, and the call waits once for the stream
  static constexpr int kPinnedHist = 1024;
  static constexpr size_t kPinnedScal = (sizeof(tc::DevScalars) + 63) / 64 * 64;
  unsigned char *h_step = nullptr;
  // the device scalars and, kPinnedScal bytes after them in the same
  // allocation, the step history of up to kPinnedHist steps, so that tc_step
  // reads both with one copy; dt_hist_own: the history outgrew it and has an
  // allocation of its own
  bool dt_hist_own = false;
  double *LP, *UP, *LH, *UH, *LT, *UT, *infl, *Ainv;
  double *dt_hist;
  int dt_hist_cap = 0;
  double *diag_part, *diag_out;
  tc::DevScalars *scal;
  tc::NLParams nl, nl32;
  int precision = 0;            // 0: FP64 everywhere; 1: FP32 transforms/products
  double *prof = nullptr;       // mean-flow profile for the mixed path
  float2 *X32 = nullptr;        // mixed path: FP32 copy of the perturbation state
  size_t smem32_zinv = 0, smem32_theta = 0, smem32_zfwd = 0;
  // adjoint buffers (allocated on first use)
  double2 *Va = nullptr, *Gdr = nullptr, *Rb = nullptr, *Ybar = nullptr, *Nb = nullptr,
          *Xb = nullptr, *Phys = nullptr;
  size_t smem_adj_zinv = 0, smem_adj_theta = 0, smem_adj_zfwd = 0;
  double ic_su = 0.0, ic_sT = 0.0;   // scales frozen by tc_init_perturbation
  tc::LinParams lin;
  size_t smem_zinv, smem_theta, smem_zfwd;
  long long launches = 0;        // kernels launched since tc_create
  int timing = 0;
  int capturing = 0;            // a graph is capturing this context's stream
  int tile_mb = 0, tile_lb = 0, tile_mbf = 0;   // nonlinear-stage tile overrides (0: default)
  int tile_mb_adj = 0;          // m columns per CTA of the adjoint's axial kernels (0: default)
  int n_corr = 1;               // corrector passes per step
  // azimuthal transforms on the tensor cores (theta_tc.cu): the DFT matrix's
  // BF16 slices (device, null when the size is not supported) and the option
  unsigned char *d_dft_tc = nullptr;
  int tensor_theta = 0;
  // inverse axial transforms on the tensor cores (zinv_tc.cu): the folded
  // axial DFT matrix's BF16 slices (device, null when not supported) and the
  // option
  unsigned char *d_dft_ztc = nullptr;
  int tensor_z = 0;
  int flux = 0;                 // axial-flux constraint on the (0,0) u_z mode
  double eps_c = 0.0;           // centrifugal buoyancy coefficient
  double *flux_ug = nullptr;    // device (Nr): unit-forcing response of the (0,0) u_z operator
  // one step captured as a CUDA graph and replayed by tc_step (timing off)
  int use_graph = 1;
  long long gen = 0;            // bumped whenever a launch parameter may change
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  long long graph_gen = -1;
  double graph_dt = 0.0;
  long long graph_launches = 0; // kernels in one replay
  // recorded-segment graphs (tc_step_record, tc_adjoint_steps), keyed by
  // their buffers, length, step and the generation counter
  struct CachedGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long gen = -1, launches = 0;
    const void *a = nullptr, *b = nullptr;
    int n = 0;
    double dt = 0.0;
  } rec_graph, adj_graph;
  tc::KernelTimer timers[tc::KNUM];
};

namespace tc {
// Brackets one kernel launch: counts it and, with timing on, records a pair
// of events on the context's stream around it.
struct LaunchScope {
  tc_ctx *c;
  int id;
  LaunchScope(tc_ctx *c_, int id_);
  ~LaunchScope();
};
}  // namespace tc

namespace tc {

// The dynamic shared-memory limit is a property of the kernel function, shared
// by every context of the process, so each kernel is opened up to the
// device's opt-in maximum instead of one context's own need (a smaller launch
// is unaffected by the larger limit).
template <typename F>
inline void allow_smem(F *kernel) {
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) mx -= (int)fa.sharedSizeBytes;
  if (mx > 0) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

// tc_host.cu
// True when `extra` more device bytes would take the context past its
// memory budget (option "memory_budget").
inline bool over_budget(const tc_ctx *c, size_t extra) {
  return c->mem_budget && c->device_bytes + extra > c->mem_budget;
}
void enqueue_step(tc_ctx *c, double dt_fixed, int step_index);
tc_status commit_staged_state(tc_ctx *c);   // Xp -> X after validation
cudaError_t ensure_step_graph(tc_ctx *c, double dt_fixed);

// nonlinear.cu
void launch_nonlinear(tc_ctx *c, const double2 *X, double2 *N, unsigned long long *rate_bits,
                      int mode, double2 *phys_out = nullptr);
void setup_nonlinear(tc_ctx *c);

// linear.cu
void launch_factor_poisson(tc_ctx *c);
void launch_refactor(tc_ctx *c);
void launch_dt_policy(tc_ctx *c, double dt_fixed, int step_index);
void launch_rhs(tc_ctx *c, const double2 *X, const double2 *N0);
void invalidate_rhs_identity(tc_ctx *c);   // enqueued on the context's stream
// Xprev (nullable): previous iterate; the stage then records max |Xout - Xprev|.
void launch_stage(tc_ctx *c, const double2 *N, double2 *Xout, double2 *Pout,
                  const double2 *Xprev = nullptr);
void launch_check_finite(tc_ctx *c, const double2 *X, long long n);
void launch_state_check(tc_ctx *c, const double2 *X);
void setup_linear(tc_ctx *c);
void launch_stage_adjoint(tc_ctx *c, const double2 *Lb, double2 *Rb);
void launch_stage_split_adjoint(tc_ctx *c, const double2 *Rb, double2 *Ybar, double2 *Nb,
                                int accumulate);
void launch_rhs_adjoint(tc_ctx *c, const double2 *Ybar, double2 *Xb, double2 *Nb);
void launch_herm_project(tc_ctx *c, double2 *X);
void launch_objective_grad(tc_ctx *c, const double2 *X, double2 *G);
void setup_nonlinear_adjoint(tc_ctx *c);
// phys_in (nullable): the forward physical fields of X written by
// launch_nonlinear(..., phys_out) on the same X.
void launch_nonlinear_adjoint(tc_ctx *c, const double2 *X, const double2 *Nb, double2 *Xb,
                              int accumulate, const double2 *phys_in = nullptr);
void launch_symmetrise(tc_ctx *c, double2 *X);

// diag.cu
void launch_diagnostics(tc_ctx *c);

// theta_tc.cu: the inverse azimuthal transforms of the FP64 nonlinear stage
// as BF16 slice products on the tensor cores (FP64-accurate), then the
// products and the forward transform as in k_theta
bool theta_tc_supported(const Sizes &s);
size_t theta_tc_table_bytes();
void build_theta_dft(int Nt, int M, std::vector<unsigned short> &out);
void setup_theta_tc();
// Encode the TMA tensor map of V for k_theta_tc into map (128 bytes, 64-byte
// aligned); false if the driver refuses it (the caller runs k_theta instead).
bool theta_tc_map(void *map, const double2 *V, const Sizes &s);
// arm = false (test hook "selftest_no_copy"): the DFT chunk copies never
// start, so each CTA's first wait runs out and the timeout flag is set.
void launch_theta_tc(cudaStream_t st, const void *map, double2 *W, const NLParams &p,
                     const unsigned char *dft, unsigned long long *rate_bits, int *timeout,
                     bool arm);

// zinv_tc.cu: the inverse axial transforms of the FP64 nonlinear stage (with
// the d/dr stencil and the z derivative) as BF16 slice products of the folded
// axial DFT matrix on the tensor cores (FP64-accurate); writes V as k_zinv
bool zinv_tc_supported(const Sizes &s);
size_t zinv_tc_table_bytes();
void build_zinv_dft(int Nz, int K, std::vector<unsigned short> &out);
void setup_zinv_tc();
// arm = false (test hook "selftest_no_copy"): the matrix chunk copies never
// start, so each CTA's first wait runs out and the timeout flag is set.
void launch_zinv_tc(cudaStream_t st, const double2 *X, double2 *V, const NLParams &p,
                    const unsigned char *dft, int *timeout, bool arm);

}  // namespace tc
