// Ensemble of independent runs of uneven size on one GPU (batching form).
//
// Each member is an ordinary context.  Two ways to step them all:
//   mode 0 (default): one step of every member captured once into a CUDA
//     graph, the members as independent branches between a fork and a join,
//     replayed once per step;
//   mode 1: one persistent kernel (k_ensemble) runs every step of every
//     member; work items are single CTA tiles of the step's kernels, and each
//     member advances through its stages on its own.
// Mode 0 is the default because it is faster: the persistent kernel is one
// function compiled for the register demand of its largest body (128 per
// thread, 16 warps per SM), while the members' own kernels run at 24 to 64
// warps per SM, and its sweep tiles leave half of a CTA idle.
// Both run exactly the arithmetic of the member stepped alone.
//
// Tiles: before the first step, each size class (Nr, Ntheta, Nz, fields,
// precision) is tuned once by timing the nonlinear stage for candidate tile
// shapes (m columns per CTA of the axial kernels, z rows per CTA of the
// azimuthal kernel) and keeping the fastest; the persistent kernel then
// shrinks any tile whose shared memory exceeds its per-CTA budget.  Tiles do
// not change the arithmetic, so results are bit-identical for every choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "lin_body.cuh"
#include "nl_body.cuh"
#include "tc_internal.h"

struct tc_ens {
  std::vector<tc_ctx *> m;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t s0 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double> graph_dt;
  std::vector<long long> graph_gen;   // members' launch-parameter generations at capture
  // persistent launch (mode 1): member table, item offsets, grid-barrier state
  int mode = 0;
  void *d_mem = nullptr;       // EnsMember[n] (device)
  int *d_ntiles = nullptr;     // tiles [n][stage] (device)
  unsigned *d_sched = nullptr; // stage [n], claim and done [n][G] of one launch (device)
  int *d_fail = nullptr;       // failure flag of the last launch (device)
  size_t smem = 0;
  int grid = 0;
  std::vector<double> plan_dt;
  std::vector<long long> plan_gen;
  long long items_per_step = 0;
};

namespace tc {
namespace {

using ClassKey = std::tuple<int, int, int, int, int>;

ClassKey class_of(const tc_ctx *c) {
  return ClassKey(c->sz.Nr, c->sz.Nt, c->sz.Nz, c->sz.nf, c->precision);
}

// Mean time of the nonlinear stage with the context's current tiles.
float time_nonlinear(tc_ctx *c, cudaEvent_t a, cudaEvent_t b, int reps) {
  launch_nonlinear(c, c->X, c->N0, nullptr, 0);   // warm-up
  cudaEventRecord(a, c->stream);
  for (int r = 0; r < reps; ++r) launch_nonlinear(c, c->X, c->N0, nullptr, 0);
  cudaEventRecord(b, c->stream);
  cudaEventSynchronize(b);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  return ms / reps;
}

// Coordinate search over the axial tile (MB), then the azimuthal tile (LB).
tc_status autotune(tc_ctx *c, int *best_mb, int *best_lb) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return TC_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return TC_ERR_CUDA;
  }
  // widths that are not powers of two change how the grids fill the 152 SMs
  const int cand_mb[] = {1, 2, 3, 4, 5, 6, 8};
  const int cand_lb[] = {1, 2, 3, 4, 8};
  // the forward axial kernel's width stays at its default while tile_mb is
  // searched, so that search sees only the inverse kernel change
  tc_set_option(c, "tile_mbf", (c->precision == 1) ? c->nl32.MBf : c->nl.MBf);
  tc_set_option(c, "tensor_theta", 0);
  tc_set_option(c, "tensor_z", 0);
  float best = 1e30f;
  int bm = 0;
  for (int mb : cand_mb) {
    if (mb > c->sz.NM) break;
    if (tc_set_option(c, "tile_mb", mb) != TC_OK) continue;
    const float t = time_nonlinear(c, a, b, 3);
    if (t < best) {
      best = t;
      bm = mb;
    }
  }
  if (bm) tc_set_option(c, "tile_mb", bm);
  best = 1e30f;
  int bl = 0;
  for (int lb : cand_lb) {
    if (tc_set_option(c, "tile_lb", lb) != TC_OK) continue;
    const float t = time_nonlinear(c, a, b, 3);
    if (t < best) {
      best = t;
      bl = lb;
    }
  }
  if (bl) tc_set_option(c, "tile_lb", bl);
  // the azimuthal stage on the tensor cores, where it applies, against the
  // FFT kernel with the tile just chosen
  if (c->precision == 0 && c->d_dft_tc) {
    tc_set_option(c, "tensor_theta", 1);
    const float t = time_nonlinear(c, a, b, 3);
    if (t >= best) tc_set_option(c, "tensor_theta", 0);
    else best = t;
  }
  // the inverse axial stage on the tensor cores, where it applies, against
  // the FFT kernel with the choices made so far
  if (c->precision == 0 && c->d_dft_ztc) {
    tc_set_option(c, "tensor_z", 1);
    if (time_nonlinear(c, a, b, 3) >= best) tc_set_option(c, "tensor_z", 0);
  }
  // the forward axial kernel's own width (its grid fills the SMs differently)
  best = 1e30f;
  int bf = 0;
  for (int mb : cand_mb) {
    if (mb > c->sz.NM) break;
    if (tc_set_option(c, "tile_mbf", mb) != TC_OK) continue;
    const float t = time_nonlinear(c, a, b, 3);
    if (t < best) {
      best = t;
      bf = mb;
    }
  }
  if (bf) tc_set_option(c, "tile_mbf", bf);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    std::fprintf(stderr, "libtc: autotune: %s\n", cudaGetErrorString(err));
    return TC_ERR_CUDA;
  }
  *best_mb = bm;
  *best_lb = bl;
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Persistent ensemble kernel (mode 1).
//
// One launch runs a chunk of steps of every member.  Each member's step is
// the fixed sequence of stages of enqueue_step (n_corr = 1), and every stage
// is a set of work items, one CTA tile of that stage's kernel each.  The
// members advance independently: member m's stage counter g (a global stage
// index over the chunk's steps) moves to g + 1 when the last tile of stage g
// is done, and a CTA looking for work scans the members (one lane of warp 0
// per member) for one whose current stage still has unclaimed tiles, claims
// the next tile with an atomic counter and runs it.  Nothing waits on a
// dependency: a tile is only claimed once its stage is current, i.e. once
// every earlier stage of its member is complete, so latency-bound stages of
// one member (the radial sweeps) overlap with the transforms of others, as
// independent kernels would.  A CTA that finds no ready work sleeps and scans
// again; if that lasts kEnsIdleNs it raises the failure flag, every CTA
// leaves, and tc_ensemble_step reports TC_ERR_TIMEOUT (a stage that is never
// published -- the test hook -- ends that way, without a fault).  Each tile
// runs the same device body as the member's own kernel.
enum EnsKind : int {
  EK_PREP, EK_ZINV, EK_THETA, EK_ZFWD, EK_DT, EK_FACTH, EK_INFL, EK_RHS, EK_PRHS, EK_SWEEP_P,
  EK_HRHS, EK_SWEEP_H, EK_ALPHA, EK_CORRECT
};
struct EnsStageDef {
  int kind, pass;   // pass 0: predictor (X -> Xp, with N0), 1: corrector (Xp -> X, with N1)
};
__constant__ EnsStageDef c_ens_stages[] = {
    {EK_PREP, 0},  {EK_ZINV, 0},    {EK_THETA, 0}, {EK_ZFWD, 0},    {EK_DT, 0},
    {EK_FACTH, 0}, {EK_INFL, 0},    {EK_RHS, 0},   {EK_PRHS, 0},    {EK_SWEEP_P, 0},
    {EK_HRHS, 0},  {EK_SWEEP_H, 0}, {EK_ALPHA, 0}, {EK_CORRECT, 0}, {EK_PREP, 1},
    {EK_ZINV, 1},  {EK_THETA, 1},   {EK_ZFWD, 1},  {EK_PRHS, 1},    {EK_SWEEP_P, 1},
    {EK_HRHS, 1},  {EK_SWEEP_H, 1}, {EK_ALPHA, 1}, {EK_CORRECT, 1}};
constexpr int kEnsStages = 24;
const int h_ens_kind[kEnsStages] = {EK_PREP,  EK_ZINV,  EK_THETA,   EK_ZFWD,  EK_DT,
                                    EK_FACTH, EK_INFL,  EK_RHS,     EK_PRHS,  EK_SWEEP_P,
                                    EK_HRHS,  EK_SWEEP_H, EK_ALPHA, EK_CORRECT, EK_PREP,
                                    EK_ZINV,  EK_THETA, EK_ZFWD,    EK_PRHS,  EK_SWEEP_P,
                                    EK_HRHS,  EK_SWEEP_H, EK_ALPHA, EK_CORRECT};
constexpr int kEnsThreads = 256;
constexpr int kEnsSweepGroups = 2;    // sweep tiles per item, 64 threads each
constexpr int kEnsSweepStages = 2;    // factor ring depth of those tiles
constexpr size_t kEnsSweepRing = sizeof(double) * kEnsSweepStages * kSweepStageDoubles;
constexpr size_t kEnsSweepGroupBytes = kEnsSweepRing + 64;   // + mbarriers and abort flag
constexpr size_t kEnsSmemBudget = 110 * 1024;   // two CTAs per SM
constexpr long long kEnsIdleNs = 2000000000LL;   // 2 s without ready work
constexpr int kEnsMaxChunk = 50;                   // steps per launch

// Launch parameters of one member (device copy; see ens_item).
struct EnsMember {
  NLParams nl[2];     // transform parameters of the two passes (mixed: Xfull differs)
  LinParams lin;
  SweepArgs swP, swH;
  double2 *X, *Xp, *N0, *N1, *Yb, *P, *alpha;
  void *V, *W;
  double *Ps, *U, *UT, *prof;
  float2 *X32;
  float *prof32;
  DevScalars *sc;
  double dt, cfl, dt_max;
  int mixed, nmb, nlb, nmbf, nprx, nprof, nsw_p, nsw_h, swx;
};

// Scheduler state of one launch (zeroed before it): per member its current
// global stage, and per (member, global stage) the claimed and done tiles.
struct EnsSched {
  unsigned *stage;   // [n]
  unsigned *claim;   // [n][G]
  unsigned *done;    // [n][G]
};

struct GroupSync {
  int id;   // named barrier of one 64-thread group
  __device__ void operator()() const {
    asm volatile("bar.sync %0, 64;" :: "r"(id) : "memory");
  }
};

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) {
  return *reinterpret_cast<const volatile unsigned *>(p);
}

// Tiles per claim, by stage kind: a claim covers that many consecutive tiles
// (the scan and the counters cost about as much as a small tile).
__constant__ int c_ens_batch[] = {8, 4, 2, 4, 1, 1, 1, 8, 2, 1, 8, 1, 8, 8};
const int h_ens_batch[] = {8, 4, 2, 4, 1, 1, 1, 8, 2, 1, 8, 1, 8, 8};

// Tiles of a stage kind for one member (one CTA tile of that kind's kernel
// each; the sweeps count tile pairs).
__host__ __device__ __forceinline__ int ens_tiles(const EnsMember &m, int kind) {
  const Sizes &s = m.lin.sz;
  auto cd = [](long long a, long long b) { return (int)((a + b - 1) / b); };
  switch (kind) {
    case EK_PREP: return m.mixed ? m.nprof + cd((long long)s.nf * s.S, kEnsThreads) : 0;
    case EK_ZINV: return m.nmb * s.Nr * s.nf;
    case EK_THETA: return m.nlb * s.Nr;
    case EK_ZFWD: return m.nmbf * s.Nr;
    case EK_DT: return 1;
    case EK_FACTH: return cd(m.lin.nopH + m.lin.nopT, kEnsThreads);
    case EK_INFL: return cd(m.lin.nopP, kEnsThreads);
    case EK_RHS:
    case EK_HRHS:
    case EK_CORRECT: return cd(s.S, kEnsThreads);
    case EK_PRHS: return m.nprx * cd(s.Nr, kPrL);
    case EK_SWEEP_P: return cd(m.nsw_p, kEnsSweepGroups);
    case EK_SWEEP_H: return cd(m.nsw_h, kEnsSweepGroups);
    case EK_ALPHA: return cd(2LL * s.nmode, kEnsThreads);
  }
  return 0;
}

// One tile: tile `t` of stage `d` of member `m`.
__device__ __forceinline__ void ens_item(const EnsMember &m, EnsStageDef d, int t,
                                         unsigned char *smem) {
  const Sizes &s = m.lin.sz;
  const int tid = threadIdx.x;
  const long long i = (long long)t * kEnsThreads + tid;
  const NLParams &p = m.nl[d.pass];
  const double2 *Xin = d.pass ? m.Xp : m.X;
  double2 *Nout = d.pass ? m.N1 : m.N0;
  switch (d.kind) {
    case EK_PREP:
      if (t < m.nprof) meanprof_body(Xin, m.prof, m.prof32, s, m.lin.rad, t * kEnsThreads + tid);
      else tofloat_body(Xin, m.X32, s, (long long)(t - m.nprof) * kEnsThreads + tid);
      break;
    case EK_ZINV: {
      const int bx = t % m.nmb, r = t / m.nmb;
      if (m.mixed)
        zinv_body<float>(m.X32, static_cast<float2 *>(m.V), p, smem, bx, r % s.Nr, r / s.Nr);
      else
        zinv_body<double>(Xin, static_cast<double2 *>(m.V), p, smem, bx, r % s.Nr, r / s.Nr);
      break;
    }
    case EK_THETA: {
      unsigned long long *rate = d.pass ? nullptr : &m.sc->rate_bits;
      if (m.mixed)
        theta_body<float>(static_cast<const float2 *>(m.V), static_cast<float2 *>(m.W), p, rate,
                          m.sc->norm_bits, 0, smem, t % m.nlb, t / m.nlb);
      else
        theta_body<double>(static_cast<const double2 *>(m.V), static_cast<double2 *>(m.W), p,
                           rate, m.sc->norm_bits, 0, smem, t % m.nlb, t / m.nlb);
      break;
    }
    case EK_ZFWD:
      if (m.mixed)
        zfwd_body<float>(static_cast<const float2 *>(m.W), Nout, p, smem, t % m.nmbf,
                         t / m.nmbf);
      else
        zfwd_body<double>(static_cast<const double2 *>(m.W), Nout, p, smem, t % m.nmbf,
                          t / m.nmbf);
      break;
    case EK_DT:
      if (tid == 0) dt_policy_body(m.sc, m.dt, m.cfl, m.dt_max, nullptr, 0);
      break;
    case EK_FACTH:
      factor_helm_body(m.lin, m.sc, (int)i);
      break;
    case EK_INFL:
      influence_body(m.lin, m.sc, (int)i);
      break;
    case EK_RHS:
      rhs_body(m.X, m.N0, m.Yb, m.N1, m.P, m.lin, m.sc, i);
      break;
    case EK_PRHS:
      prhs_body(m.Yb, Nout, m.Ps, m.UT, m.lin, reinterpret_cast<double2 *>(smem), t % m.nprx,
                t / m.nprx);
      break;
    case EK_SWEEP_P:
    case EK_SWEEP_H: {
      const int grp = tid >> 6;
      const int nt = d.kind == EK_SWEEP_P ? m.nsw_p : m.nsw_h;
      const int u = t * kEnsSweepGroups + grp;
      if (grp < kEnsSweepGroups && u < nt) {
        unsigned char *base = smem + grp * kEnsSweepGroupBytes;
        unsigned long long *bars = reinterpret_cast<unsigned long long *>(base + kEnsSweepRing);
        int *abort_flag = reinterpret_cast<int *>(bars + kEnsSweepStages);
        const int bx = u % m.swx, r = u / m.swx;
        sweep_body<false, kEnsSweepStages>(d.kind == EK_SWEEP_P ? m.swP : m.swH, m.sc, bx,
                                           r % s.NM, r / s.NM, tid & 63,
                                           reinterpret_cast<double *>(base), bars, abort_flag,
                                           GroupSync{1 + grp});
      }
      break;
    }
    case EK_HRHS:
      hrhs_body(m.Yb, Nout, m.Ps, m.U, m.lin, i);
      break;
    case EK_ALPHA:
      alpha_body(m.U, m.alpha, m.lin, i);
      break;
    case EK_CORRECT:
      if (d.pass) correct_body(m.U, m.Ps, m.alpha, m.X, m.P, m.Xp, m.lin, m.sc, i);
      else correct_body(m.U, m.Ps, m.alpha, m.Xp, m.P, nullptr, m.lin, m.sc, i);
      break;
  }
}

__global__ void __launch_bounds__(kEnsThreads, 2)
k_ensemble(const EnsMember *__restrict__ mem, const int *__restrict__ ntiles, int nmem,
           int nsteps, EnsSched sch, int *fail, int selftest) {
  extern __shared__ __align__(128) unsigned char ens_smem[];
  __shared__ int pick_m, pick_t;
  __shared__ unsigned pick_g;
  const unsigned G = (unsigned)nsteps * kEnsStages;
  int start = blockIdx.x % nmem;          // first member this CTA looks at (warp 0, uniform)
  unsigned long long idle_since = 0ull;   // thread 0: start of the current idle spell
  while (true) {
    if (threadIdx.x < 32) {
      // warp 0 scans 32 members at a time for a current stage with tiles left
      const int lane = threadIdx.x;
      int found = -1, nfin = 0;
      unsigned fg = 0u, ft = 0u;
      for (int base = 0; base < nmem && found < 0; base += 32) {
        const int k = base + lane;
        int m = 0, nt = 0;
        unsigned g = 0u;
        bool cand = false, fin = false;
        if (k < nmem) {
          m = (start + k) % nmem;
          g = ld_volatile(&sch.stage[m]);
          if (g >= G) {
            fin = true;
          } else {
            nt = ntiles[m * kEnsStages + (int)(g % kEnsStages)];
            if (nt == 0) atomicCAS(&sch.stage[m], g, g + 1u);   // an empty stage passes at once
            else cand = ld_volatile(&sch.claim[(size_t)m * G + g]) < (unsigned)nt;
          }
        }
        nfin += __popc(__ballot_sync(0xffffffffu, fin));
        unsigned mask = __ballot_sync(0xffffffffu, cand);
        while (mask && found < 0) {   // try the candidates in lane order
          const int l = __ffs(mask) - 1;
          unsigned t = 0u;
          if (lane == l) t = atomicAdd(&sch.claim[(size_t)m * G + g], 1u);
          t = __shfl_sync(0xffffffffu, t, l);
          const int ntl = __shfl_sync(0xffffffffu, nt, l);
          if (t < (unsigned)ntl) {
            found = __shfl_sync(0xffffffffu, m, l);
            fg = __shfl_sync(0xffffffffu, g, l);
            ft = t;
          }
          mask &= mask - 1u;
        }
      }
      if (found >= 0) start = found;   // every lane: the next scan starts there
      if (lane == 0) {
        __threadfence();   // acquire: the claimed stage's inputs are complete
        pick_m = found >= 0 ? found : (nfin == nmem ? -2 : -1);
        pick_g = fg;
        pick_t = (int)ft;
        if (found >= 0) {
          idle_since = 0ull;
        } else if (nfin < nmem) {
          const unsigned long long now = global_ns();
          if (idle_since == 0ull) idle_since = now;
          if (*reinterpret_cast<volatile int *>(fail) ||
              (long long)(now - idle_since) > kEnsIdleNs) {
            atomicExch(fail, 1);
            pick_m = -2;
          } else {
            __nanosleep(256);
          }
        }
      }
    }
    __syncthreads();
    const int m = pick_m;
    if (m == -2) break;
    if (m >= 0) {
      const unsigned g = pick_g;
      const EnsStageDef d = c_ens_stages[g % kEnsStages];
      const int B = c_ens_batch[d.kind];
      const int t1 = min((pick_t + 1) * B, ens_tiles(mem[m], d.kind));
      for (int t = pick_t * B; t < t1; ++t) {
        ens_item(mem[m], d, t, ens_smem);
        __syncthreads();   // the tile's shared memory is free for the next one
      }
      if (threadIdx.x == 0) {
        __threadfence();   // release: this tile's results before the count
        const unsigned nt = (unsigned)ntiles[m * kEnsStages + (int)(g % kEnsStages)];
        const unsigned d = atomicAdd(&sch.done[(size_t)m * G + g], 1u) + 1u;
        // test hook: member 0's first transform stage (global stage 1, never
        // empty) is never published
        const bool hold = selftest && m == 0 && g == 1u;
        if (d == nt && !hold) {
          __threadfence();
          atomicExch(&sch.stage[m], g + 1u);
        }
      }
    }
    __syncthreads();   // pick_* is rewritten by the next scan
  }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

SweepArgs sweep_args_of(const tc_ctx *c) {
  SweepArgs a{};
  a.Nr = c->sz.Nr;
  a.Nrp = c->lin.Nrp;
  a.K = c->sz.K;
  a.NK = c->sz.NK;
  a.nmode = c->sz.nmode;
  a.S = c->sz.S;
  a.arm = 1;
  return a;
}

// Claims of stage kind k for one member (host): its tiles in batches.
int ens_items(const EnsMember &m, int k) {
  const int tiles = ens_tiles(m, k);
  return (tiles + h_ens_batch[k] - 1) / h_ens_batch[k];
}

// Largest transform-tile shared memory of a context in its precision.
size_t transform_smem(const tc_ctx *c) {
  return c->precision == 1 ? std::max({c->smem32_zinv, c->smem32_theta, c->smem32_zfwd})
                           : std::max({c->smem_zinv, c->smem_theta, c->smem_zfwd});
}

// Shrink a member's tiles until they fit the persistent kernel's budget
// (tiles do not change the arithmetic).
void fit_tiles(tc_ctx *c, size_t budget) {
  for (int guard = 0; guard < 64 && transform_smem(c) > budget; ++guard) {
    const NLParams &q = (c->precision == 1) ? c->nl32 : c->nl;
    const size_t zi = c->precision == 1 ? c->smem32_zinv : c->smem_zinv;
    const size_t th = c->precision == 1 ? c->smem32_theta : c->smem_theta;
    if (th > budget && q.LB > 1) tc_set_option(c, "tile_lb", q.LB - 1);
    else if (zi > budget && q.MB > 1) tc_set_option(c, "tile_mb", q.MB - 1);
    else if (q.MBf > 1) tc_set_option(c, "tile_mbf", q.MBf - 1);
    else break;
  }
}

void drop_plan(tc_ens *e) {
  if (e->d_mem) cudaFree(e->d_mem);
  if (e->d_ntiles) cudaFree(e->d_ntiles);
  if (e->d_sched) cudaFree(e->d_sched);
  if (e->d_fail) cudaFree(e->d_fail);
  e->d_mem = nullptr;
  e->d_ntiles = nullptr;
  e->d_sched = nullptr;
  e->d_fail = nullptr;
  e->plan_dt.clear();
  e->plan_gen.clear();
}

// Member table and tile counts for the persistent kernel (rebuilt when a
// member's step or launch parameters change).
tc_status build_plan(tc_ens *e, const double *dt) {
  const int n = (int)e->m.size();
  drop_plan(e);
  std::vector<EnsMember> mem(n);
  size_t smem = std::max<size_t>((size_t)kPrWin * kPrW * sizeof(double2),
                                 kEnsSweepGroups * kEnsSweepGroupBytes);
  for (int i = 0; i < n; ++i) {
    tc_ctx *c = e->m[i];
    if (c->n_corr != 1 || c->flux || c->selftest_no_copy) return TC_ERR_UNSUPPORTED;
    fit_tiles(c, kEnsSmemBudget);
    if (transform_smem(c) > kEnsSmemBudget) return TC_ERR_UNSUPPORTED;
    smem = std::max(smem, transform_smem(c));
    const Sizes &s = c->sz;
    EnsMember &m = mem[i];
    m.mixed = c->precision == 1;
    for (int pass = 0; pass < 2; ++pass) {
      NLParams q = m.mixed ? c->nl32 : c->nl;
      if (m.mixed) {
        q.mixed = 1;
        q.Xfull = pass ? c->Xp : c->X;
        q.prof = c->prof;
      }
      q.phys_out = nullptr;
      m.nl[pass] = q;
    }
    const NLParams &q = m.nl[0];
    m.lin = c->lin;
    double *U = reinterpret_cast<double *>(c->U0);
    m.U = U;
    m.UT = (s.nf == 4) ? U + 6 * s.S : nullptr;
    m.swP = sweep_args_of(c);
    m.swP.f[0] = SweepField{c->lin.LP, c->lin.UP, c->Ps, 0, 1, c->lin.nopP};
    if (m.UT) m.swP.f[1] = SweepField{c->lin.LT, c->lin.UT, m.UT, 0, 0, c->lin.nopT};
    m.swH = sweep_args_of(c);
    m.swH.f[0] = SweepField{c->lin.LH, c->lin.UH, U + 0 * s.S, +1, 0, c->lin.nopH};
    m.swH.f[1] = SweepField{c->lin.LH, c->lin.UH, U + 2 * s.S, -1, 0, c->lin.nopH};
    m.swH.f[2] = SweepField{c->lin.LH, c->lin.UH, U + 4 * s.S, 0, 0, c->lin.nopH};
    m.X = c->X;
    m.Xp = c->Xp;
    m.N0 = c->N0;
    m.N1 = c->N1;
    m.Yb = c->Yb;
    m.P = c->P;
    m.alpha = c->alpha_buf;
    m.V = c->V;
    m.W = c->W;
    m.Ps = c->Ps;
    m.prof = c->prof;
    m.X32 = c->X32;
    m.prof32 = c->d_prof32;
    m.sc = c->scal;
    m.dt = dt[i];
    m.cfl = c->cfl;
    m.dt_max = c->dt_max;
    m.nmb = cdiv(s.NM, q.MB);
    m.nlb = cdiv(s.Nz, q.LB);
    m.nmbf = cdiv(s.NM, q.MBf);
    m.nprx = cdiv(s.nmode, kPrW);
    m.nprof = cdiv(s.Nr, kEnsThreads);
    m.swx = (s.K + kSweepOps) / kSweepOps;
    m.nsw_p = m.swx * s.NM * (m.UT ? 2 : 1);
    m.nsw_h = m.swx * s.NM * 3;
  }
  std::vector<int> ntiles((size_t)n * kEnsStages, 0);
  long long items = 0;
  for (int i = 0; i < n; ++i)
    for (int st = 0; st < kEnsStages; ++st) {
      ntiles[(size_t)i * kEnsStages + st] = ens_items(mem[i], h_ens_kind[st]);
      items += ntiles[(size_t)i * kEnsStages + st];
    }
  e->items_per_step = items;
  // kernel attributes and a grid of every CTA that can be resident
  if (cudaFuncSetAttribute(k_ensemble, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_UNSUPPORTED;
  }
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ensemble, kEnsThreads, smem) !=
          cudaSuccess || per < 1) {
    cudaGetLastError();
    return TC_ERR_UNSUPPORTED;
  }
  e->grid = nsm * per;
  e->smem = smem;
  const size_t words = (size_t)n * (1 + 2 * (size_t)kEnsMaxChunk * kEnsStages);
  if (cudaMalloc(&e->d_mem, sizeof(EnsMember) * n) != cudaSuccess ||
      cudaMalloc(&e->d_ntiles, sizeof(int) * ntiles.size()) != cudaSuccess ||
      cudaMalloc(&e->d_sched, sizeof(unsigned) * words) != cudaSuccess ||
      cudaMalloc(&e->d_fail, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    drop_plan(e);
    return TC_ERR_OOM;
  }
  if (cudaMemcpy(e->d_mem, mem.data(), sizeof(EnsMember) * n, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(e->d_ntiles, ntiles.data(), sizeof(int) * ntiles.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    drop_plan(e);
    return TC_ERR_CUDA;
  }
  e->plan_dt.assign(dt, dt + n);
  e->plan_gen.resize(n);
  for (int i = 0; i < n; ++i) e->plan_gen[i] = e->m[i]->gen;
  return TC_OK;
}

// nsteps steps of every member in one cooperative launch on e->s0.
// selftest != 0: member 0's first transform stage is never published
// (test hook of the bounded idle wait: the other members finish, then every
// CTA runs out of ready work, and the step reports TC_ERR_TIMEOUT).
tc_status persistent_steps(tc_ens *e, int nsteps, const double *dt, int selftest) {
  const int n = (int)e->m.size();
  bool same = e->d_mem && (int)e->plan_dt.size() == n &&
              std::equal(e->plan_dt.begin(), e->plan_dt.end(), dt);
  for (int i = 0; same && i < n; ++i) same = e->plan_gen[i] == e->m[i]->gen;
  if (!same) {
    const tc_status st = build_plan(e, dt);
    if (st != TC_OK) return st;
  }
  if (cudaMemsetAsync(e->d_fail, 0, sizeof(int), e->s0) != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_CUDA;
  }
  const EnsMember *dm = static_cast<const EnsMember *>(e->d_mem);
  for (int done = 0; done < nsteps;) {
    const int chunk = std::min(kEnsMaxChunk, nsteps - done);
    const size_t G = (size_t)chunk * kEnsStages;
    EnsSched sch{};
    sch.stage = e->d_sched;
    sch.claim = e->d_sched + n;
    sch.done = sch.claim + (size_t)n * G;
    const size_t words = (size_t)n * (1 + 2 * G);
    if (cudaMemsetAsync(e->d_sched, 0, sizeof(unsigned) * words, e->s0) != cudaSuccess) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
    k_ensemble<<<e->grid, kEnsThreads, e->smem, e->s0>>>(dm, e->d_ntiles, n, chunk, sch,
                                                         e->d_fail, selftest);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
    for (tc_ctx *c : e->m) c->launches += 1;
    done += chunk;
  }
  return TC_OK;
}

// Wait for the steps and collect the members' status flags.
tc_status finish_steps(tc_ens *e, int nsteps, const double *dt, bool persistent) {
  const int n = (int)e->m.size();
  if (cudaStreamSynchronize(e->s0) != cudaSuccess) {
    cudaGetLastError();
    for (tc_ctx *c : e->m) c->poisoned = true;
    return TC_ERR_CUDA;
  }
  tc_status worst = TC_OK;
  if (persistent) {
    int fail = 0;
    if (cudaMemcpy(&fail, e->d_fail, sizeof(fail), cudaMemcpyDeviceToHost) != cudaSuccess)
      return TC_ERR_CUDA;
    if (fail) worst = TC_ERR_TIMEOUT;
  }
  for (int i = 0; i < n; ++i) {
    tc_ctx *c = e->m[i];
    DevScalars sc;
    if (cudaMemcpy(&sc, c->scal, sizeof(sc), cudaMemcpyDeviceToHost) != cudaSuccess)
      return TC_ERR_CUDA;
    c->t += dt[i] * nsteps;
    if (sc.timeout) worst = TC_ERR_TIMEOUT;
    else if (c->check && sc.nonfinite && worst == TC_OK) worst = TC_ERR_NONFINITE;
  }
  return worst;
}

void drop_graph(tc_ens *e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->exec = nullptr;
  e->graph = nullptr;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_ensemble_destroy(tc_ens *e) {
  if (!e) return TC_OK;
  drop_graph(e);
  drop_plan(e);
  for (tc_ctx *c : e->m) tc_destroy(c);
  for (cudaStream_t s : e->streams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : e->joins) cudaEventDestroy(ev);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->s0) cudaStreamDestroy(e->s0);
  delete e;
  return TC_OK;
}

tc_status tc_ensemble_create(int n, const tc_params *p, int autotune_tiles, tc_ens **out) {
  if (!out || !p || n < 1 || n > 4096) return TC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (p[i].precision != 0 && p[i].precision != 1) return TC_ERR_ARG;
  tc_ens *e = new tc_ens();
  auto fail = [&](tc_status st) {
    tc_ensemble_destroy(e);
    return st;
  };
  if (cudaStreamCreateWithFlags(&e->s0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) != cudaSuccess) {
    std::fprintf(stderr, "libtc: ensemble: %s\n", cudaGetErrorString(cudaGetLastError()));
    return fail(TC_ERR_CUDA);
  }
  for (int i = 0; i < n; ++i) {
    tc_ctx *c = nullptr;
    tc_status st = tc_create(p[i].Nr, p[i].Ntheta, p[i].Nz, p[i].eta, p[i].Lz, p[i].Re_i,
                             p[i].Re_o, p[i].Ra, p[i].Pr, &c);
    if (st != TC_OK) return fail(st);
    e->m.push_back(c);
    if (p[i].precision) tc_set_option(c, "precision", p[i].precision);
    cudaStream_t s;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(TC_ERR_CUDA);
    e->streams.push_back(s);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(TC_ERR_CUDA);
    e->joins.push_back(ev);
    tc_set_stream(c, s);
  }
  if (autotune_tiles) {
    // tuned (tile_mb, tile_lb, tile_mbf, tensor_theta, tensor_z) per size class
    std::map<ClassKey, std::tuple<int, int, int, int, int>> tuned;
    for (tc_ctx *c : e->m) {
      const ClassKey k = class_of(c);
      auto it = tuned.find(k);
      if (it == tuned.end()) {
        int mb = 0, lb = 0;
        tc_status st = autotune(c, &mb, &lb);
        if (st != TC_OK) return fail(st);
        tuned[k] = std::make_tuple(mb, lb, c->tile_mbf, c->tensor_theta, c->tensor_z);
      } else {
        const auto [mb, lb, mbf, tt, tz] = it->second;
        if (mb) tc_set_option(c, "tile_mb", mb);
        if (lb) tc_set_option(c, "tile_lb", lb);
        if (mbf) tc_set_option(c, "tile_mbf", mbf);
        tc_set_option(c, "tensor_theta", tt);
        tc_set_option(c, "tensor_z", tz);
      }
    }
  }
  *out = e;
  return TC_OK;
}

tc_status tc_ensemble_member(tc_ens *e, int i, tc_ctx **ctx) {
  if (!e || !ctx || i < 0 || i >= (int)e->m.size()) return TC_ERR_ARG;
  *ctx = e->m[i];
  return TC_OK;
}

tc_status tc_ensemble_step(tc_ens *e, int nsteps, const double *dt) {
  if (!e || !dt || nsteps < 0) return TC_ERR_ARG;
  const int n = (int)e->m.size();
  for (int i = 0; i < n; ++i) {
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return TC_ERR_ARG;
    if (e->m[i]->poisoned) return TC_ERR_CUDA;
    if (e->m[i]->timing) tc_set_option(e->m[i], "timing", 0);
  }
  if (nsteps == 0) return TC_OK;
  bool persistent = e->mode >= 1;
  for (int i = 0; persistent && i < n; ++i)   // the persistent kernel runs the default scheme
    persistent = e->m[i]->n_corr == 1 && !e->m[i]->flux && !e->m[i]->selftest_no_copy;
  if (persistent) {
    for (int i = 0; i < n; ++i) {
      tc_ctx *c = e->m[i];
      cudaMemsetAsync(reinterpret_cast<char *>(c->scal) + offsetof(DevScalars, nonfinite), 0,
                      2 * sizeof(int), e->s0);
    }
    const tc_status st = persistent_steps(e, nsteps, dt, e->mode == 2);
    if (st != TC_OK) return st;
    return finish_steps(e, nsteps, dt, true);
  }
  bool same = e->exec && (int)e->graph_dt.size() == n &&
              std::equal(e->graph_dt.begin(), e->graph_dt.end(), dt);
  for (int i = 0; same && i < n; ++i) same = e->graph_gen[i] == e->m[i]->gen;
  if (!same) {
    drop_graph(e);
    // capture one step of every member as independent branches
    if (cudaStreamBeginCapture(e->s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return TC_ERR_CUDA;
    cudaEventRecord(e->fork, e->s0);
    for (int i = 0; i < n; ++i) {
      tc_ctx *c = e->m[i];
      cudaStreamWaitEvent(c->stream, e->fork, 0);
      c->capturing = 1;
      enqueue_step(c, dt[i], -1);
      c->capturing = 0;
      cudaEventRecord(e->joins[i], c->stream);
      cudaStreamWaitEvent(e->s0, e->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->s0, &g);
    if (ce != cudaSuccess || !g) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
    e->graph = g;
    if (cudaGraphInstantiate(&e->exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      drop_graph(e);
      return TC_ERR_CUDA;
    }
    e->graph_dt.assign(dt, dt + n);
    e->graph_gen.resize(n);
    for (int i = 0; i < n; ++i) e->graph_gen[i] = e->m[i]->gen;
  }
  for (int i = 0; i < n; ++i) {
    tc_ctx *c = e->m[i];
    cudaMemsetAsync(reinterpret_cast<char *>(c->scal) + offsetof(DevScalars, nonfinite), 0,
                    2 * sizeof(int), e->s0);
  }
  for (int s = 0; s < nsteps; ++s) {
    if (cudaGraphLaunch(e->exec, e->s0) != cudaSuccess) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
  }
  return finish_steps(e, nsteps, dt, false);
}

tc_status tc_ensemble_set_mode(tc_ens *e, int mode) {
  if (!e || mode < 0 || mode > 2) return TC_ERR_ARG;
  e->mode = mode;
  return TC_OK;
}

tc_status tc_ensemble_get_mode(const tc_ens *e, int *mode) {
  if (!e || !mode) return TC_ERR_ARG;
  *mode = e->mode;
  return TC_OK;
}

tc_status tc_autotune(tc_ctx *c, int *tile_mb, int *tile_lb) {
  if (!c) return TC_ERR_ARG;
  if (c->poisoned) return TC_ERR_CUDA;
  int mb = 0, lb = 0;
  const tc_status st = autotune(c, &mb, &lb);
  if (st != TC_OK) return st;
  if (tile_mb) *tile_mb = mb;
  if (tile_lb) *tile_lb = lb;
  return TC_OK;
}

tc_status tc_ensemble_kernels_per_step(const tc_ens *e, long long *count) {
  if (!e || !count) return TC_ERR_ARG;
  *count = 0;
  if (e->mode >= 1) {   // one persistent launch per tc_ensemble_step call (up to 50 steps)
    *count = e->d_mem ? 1 : 0;
    return TC_OK;
  }
  if (!e->graph) return TC_OK;
  size_t nodes = 0;
  if (cudaGraphGetNodes(e->graph, nullptr, &nodes) != cudaSuccess) return TC_ERR_CUDA;
  std::vector<cudaGraphNode_t> v(nodes);
  if (nodes && cudaGraphGetNodes(e->graph, v.data(), &nodes) != cudaSuccess) return TC_ERR_CUDA;
  long long k = 0;
  for (cudaGraphNode_t nd : v) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  *count = k;
  return TC_OK;
}

}  // extern "C"
