// Ensemble of independent runs of uneven size on one GPU.
//
// Each member is an ordinary context on its own stream.  One step of every
// member is captured once into a CUDA graph: the members are independent
// branches between a fork and a join, so one graph launch replays all of them
// and the GPU runs the branches concurrently, filling the SMs that a single
// small run leaves idle.  The graph is rebuilt only when a member's step or
// options change.  A persistent kernel was not used: every stage of a run
// depends on the previous one, which inside one launch would need grid-wide
// barriers on a shared GPU; graph replay removes the same per-launch host
// overhead.
//
// Tiles: before the first step, each size class (Nr, Ntheta, Nz, fields,
// precision) is tuned once by timing the nonlinear stage for candidate tile
// shapes (m columns per CTA of the axial kernels, z rows per CTA of the
// azimuthal kernel) and keeping the fastest.  Tiles do not change the
// arithmetic, so results are bit-identical for every choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

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
    // tuned (tile_mb, tile_lb, tile_mbf) per size class
    std::map<ClassKey, std::tuple<int, int, int>> tuned;
    for (tc_ctx *c : e->m) {
      const ClassKey k = class_of(c);
      auto it = tuned.find(k);
      if (it == tuned.end()) {
        int mb = 0, lb = 0;
        tc_status st = autotune(c, &mb, &lb);
        if (st != TC_OK) return fail(st);
        tuned[k] = std::make_tuple(mb, lb, c->tile_mbf);
      } else {
        const auto [mb, lb, mbf] = it->second;
        if (mb) tc_set_option(c, "tile_mb", mb);
        if (lb) tc_set_option(c, "tile_lb", lb);
        if (mbf) tc_set_option(c, "tile_mbf", mbf);
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
  if (cudaStreamSynchronize(e->s0) != cudaSuccess) {
    cudaGetLastError();
    for (tc_ctx *c : e->m) c->poisoned = true;
    return TC_ERR_CUDA;
  }
  tc_status worst = TC_OK;
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
