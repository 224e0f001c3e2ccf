// C ABI of the mlev library and the launch sequence of Algorithm 4.2.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kern_launch.h"
#include "plan.h"

using namespace mlev;

struct ProfRecHost {
  int launches = 0;
  double ms = 0.0, bytes = 0.0;
};

struct mlev_ctx {
  int device = 0;
  unsigned long long uid = 0;  // unique per context for the life of the process (never reused)
  int sm_count = 0, smem_per_sm = 0;  // device attributes (launch-shape decisions)
  Plan plan;
  std::string err;
  // plan tables are (re)uploaded when the workspace, the plan or the options change
  const void* uploaded_ws = nullptr;
  long long uploaded_version = -1;
  long long version = 0;
  // captured graph (captured on a private stream: the legacy default stream cannot capture)
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::string graph_key;
  int launches = 0;
  int graph_launches = 0;
  // plan cache: the planner runs again only when the setup or the precision changes
  long long built_version = -1;
  int built_precision = -1;
  int built_tail_nodes = -1;
  long long plan_gen = 0;  // bumped on every plan rebuild (keys the table upload)
  // profiling
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRecHost> prof;
  bool prof_valid = false;
  long long io_h2d = 0, io_d2h = 0;  // bytes copied by the current call
};

namespace {

std::atomic<unsigned long long> g_next_ctx_uid{1};

int fail(mlev_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(mlev_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MLEV_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
  } while (0)

// No C++ exception crosses the C interface: every entry point turns a host allocation
// failure into MLEV_ENOMEM and any other exception into MLEV_EINVAL.
#define MLEV_TRY try {
#define MLEV_CATCH(c)                                                         \
  }                                                                           \
  catch (const std::bad_alloc&) {                                             \
    return fail(c, MLEV_ENOMEM, "host allocation failed");                    \
  }                                                                           \
  catch (const std::exception& _ex) {                                         \
    return fail(c, MLEV_EINVAL, std::string("internal error: ") + _ex.what()); \
  }                                                                           \
  catch (...) {                                                               \
    return fail(c, MLEV_EINVAL, "internal error");                            \
  }

// Host-side fault injection for the error-path tests: MLEV_FAULT holds a comma-separated
// list of sites. Nothing here touches the GPU in a way that can fault or hang it.
//   plan_alloc  the planner's host allocation fails          -> MLEV_ENOMEM
//   h2d_copy    the copy of the plan tables to the device fails -> MLEV_ECUDA
//   kappa_nan   one staged coefficient value becomes NaN after validation, so the device
//               computation meets a non-finite value          -> MLEV_ENOCONV
bool fault_armed(const char* site) {
  const char* v = std::getenv("MLEV_FAULT");
  if (!v || !*v) return false;
  const std::string list = std::string(",") + v + ",";
  return list.find(std::string(",") + site + ",") != std::string::npos;
}

int map_plan_error(mlev_ctx* ctx, const std::string& e) {
  if (e.empty()) return MLEV_OK;
  if (e.rfind("UNSUPPORTED", 0) == 0) return fail(ctx, MLEV_EUNSUPPORTED, e);
  if (e.rfind("STATE", 0) == 0) return fail(ctx, MLEV_ESTATE, e);
  return fail(ctx, MLEV_EINVAL, e);
}

bool opts_valid(const mlev_opts* o) {
  return o && (o->precision == MLEV_PREC_FP64 || o->precision == MLEV_PREC_MIXED) && o->vcycles >= 1 &&
         o->refine_passes >= 1 && o->strip_vcycles >= 1 && o->pre_smooth >= 0 && o->post_smooth >= 0 &&
         o->pre_smooth + o->post_smooth >= 1 && o->coarse_sweeps >= 1 && o->level1_max_iter >= 1 &&
         o->level1_tol > 0 && o->rr_max_iter >= 1 && o->omega > 0 && o->omega < 2 && o->tail_nodes >= 0 &&
         o->fused >= 0 && o->fused <= 2 && o->reg_depths >= 0;
}

std::string opts_key(const mlev_opts* o) {
  char b[256];
  snprintf(b, sizeof b, "%d/%d/%d/%d/%d/%d/%d/%d/%.17g/%d/%.17g/%d/%d/%d/%d", o->precision, o->vcycles,
           o->refine_passes, o->strip_vcycles, o->pre_smooth, o->post_smooth, o->coarse_sweeps, o->level1_max_iter,
           o->level1_tol, o->rr_max_iter, o->omega, o->check_residuals, o->fused, o->tail_nodes, o->reg_depths);
  return b;
}

template <typename P>
P* at(void* base, const Span& s) {
  return reinterpret_cast<P*>(static_cast<char*>(base) + s.off);
}

// Kernel families for profiling (names reported by mlev_profile_read).
enum Fam {
  F_KAPPA, F_BAND, F_LEVEL1, F_INTERP, F_RHS, F_GATHER, F_SMOOTH, F_RESTRICT, F_PROLONG, F_COARSEST, F_ACCUM,
  F_REFINE, F_GLUE, F_STRIP_RHS, F_STRIP_UPD, F_AUG, F_RR, F_OUT, F_RESNORM, F_MG_DOWN, F_MG_UP, F_MG_TAIL,
  F_ADJ_RR, F_ADJ_FIELD, F_ADJ_GRAD, F_ADJ_LEVEL1, F_COUNT
};
const char* kFamName[F_COUNT] = {"kappa_levels", "coarse_band", "level1_lobpcg", "interp_embed", "rhs_aux",
                                 "mg_gather", "mg_smooth", "mg_restrict", "mg_prolong", "mg_coarsest",
                                 "mixed_accumulate", "mixed_refine_residual", "glue", "strip_rhs", "strip_update",
                                 "aug_inner", "rayleigh_ritz", "output", "residual_check", "mg_down_fused",
                                 "mg_up_fused", "mg_tail", "adj_rayleigh_ritz", "adj_fields",
                                 "adj_element_grad", "adj_level1"};

struct ProfRec {
  int fam;
  cudaEvent_t a, b;
  double bytes;
};

struct Launcher {
  mlev_ctx* ctx;
  const Plan& P;
  const mlev_opts& o;
  void* ws;
  cudaStream_t s;
  DevGeom G{};
  const double* kappa_src = nullptr;  // coarse or fine values on device (user or staged)
  int count = 0;
  bool profiling = false;
  std::vector<ProfRec>* recs = nullptr;
  std::vector<cudaEvent_t>* pool = nullptr;
  size_t next_ev = 0;
  // level checkpoints kept by the forward pass of mlev_grad_kappa (null: plain solve):
  // u~_k of level k at ck_ut + (k-1) B bstride, coefficients of u_{h_k} at ck_c + k B ncoef
  double* ck_ut = nullptr;
  double* ck_c = nullptr;
  double* ck_c0 = nullptr;

  const Tile* tiles_at(const TileList& t) const { return at<Tile>(ws, P.w_tiles) + t.off; }

  cudaEvent_t ev() {
    if (next_ev == pool->size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool->push_back(e);
    }
    return (*pool)[next_ev++];
  }

  // Enqueue one launch; in profiling mode bracket it with events on the stream.
  // pre-smoothing by plain Gauss-Seidel ends with the black half-sweep: black residuals vanish
  int black_zero() const { return o.pre_smooth >= 1 && o.omega == 1.0 ? 1 : 0; }
  // post-smoothing starts with a plain Gauss-Seidel black half-sweep: black nodes need no correction
  int red_only() const { return o.post_smooth >= 1 && o.omega == 1.0 ? 1 : 0; }

  template <class Fn>
  void go(Fam f, double bytes, Fn&& fn) {
    if (profiling) {
      cudaEvent_t a = ev(), b = ev();
      cudaEventRecord(a, s);
      fn();
      cudaEventRecord(b, s);
      recs->push_back(ProfRec{f, a, b, bytes});
    } else {
      fn();
    }
    count++;
  }

  // Traffic model, bytes per unknown (t = bytes of T): see the design notes.
  double kfine_extra() const { return P.kappa_kind == MLEV_KAPPA_PER_FINE_ELEM ? 48.0 : 0.0; }

  // how the coarsest grid of a job set is solved
  enum Coarse { C_SWEEPS = 0, C_DIRECT = 1, C_SMEM = 2 };

  template <typename T>
  void coarse_solve(int mode, const TileList& coarsest, T* X, T* F) {
    const double t = sizeof(T);
    if (mode == C_DIRECT) {
      T* inv = at<T>(ws, P.w_cinv);
      go(F_COARSEST, t * (double)coarsest.count * P.nd_max * P.nd_max,
         [&] { launch_coarsest_direct<T>(G, tiles_at(coarsest), coarsest.count, X, F, inv, P.nd_max, s); });
    } else if (mode == C_SMEM) {
      go(F_COARSEST, 4 * t * coarsest.unk, [&] {
        launch_coarsest_smem<T>(G, tiles_at(coarsest), coarsest.count, P.strip_coarse_nodes, X, F, o.coarse_sweeps,
                                o.omega, s);
      });
    } else {
      go(F_COARSEST, 4 * t * coarsest.unk * o.coarse_sweeps,
         [&] { launch_coarsest<T>(G, tiles_at(coarsest), coarsest.count, X, F, o.coarse_sweeps, o.omega, s); });
    }
  }

  template <typename T>
  void vcycle(const std::vector<TileList>& lists, const TileList& coarsest, T* X, T* F, int cmode) {
    const double t = sizeof(T);
    const int D = (int)lists.size() - 1;
    auto smooth = [&](int d, int color) {
      go(F_SMOOTH, (2 * t + 0.5 * kfine_extra()) * lists[d].unk,
         [&] { launch_smooth<T>(G, tiles_at(lists[d]), lists[d].count, X, F, color, o.omega, s); });
    };
    for (int d = 0; d < D; ++d) {
      for (int k = 0; k < o.pre_smooth; ++k) {
        smooth(d, 0);
        smooth(d, 1);
      }
      go(F_RESTRICT, (10 * t + 4 * kfine_extra()) * lists[d + 1].unk,
         [&] { launch_restrict<T>(G, tiles_at(lists[d + 1]), lists[d + 1].count, X, F, black_zero(), s); });
    }
    coarse_solve<T>(cmode, coarsest, X, F);
    for (int d = D - 1; d >= 0; --d) {
      go(F_PROLONG, 2.25 * t * lists[d].unk,
         [&] { launch_prolong<T>(G, tiles_at(lists[d]), lists[d].count, X, red_only(), s); });
      for (int k = 0; k < o.post_smooth; ++k) {
        smooth(d, 1);
        smooth(d, 0);
      }
    }
  }

  // One V-cycle with the fused kernels: down (smooth + restrict) on the depths above the
  // tail, the tail (rest of the cycle in shared memory, one block per job), then up.
  // the register-blocked FP32 down / up kernels replace the shared-memory ones where they apply
  // (per depth: the grids of a depth share one level, read from the depth's first tile)
  template <typename T>
  bool use_reg(const std::vector<TileList>* rl, int d) const {
    if (sizeof(T) != 4 || !rl || (*rl)[d].count == 0) return false;
    const int level = P.grids[P.tiles[(*rl)[d].off].grid].level;
    return rkernels_support(P.kappa_kind, level, o.pre_smooth, o.post_smooth, o.omega);
  }

  template <typename T>
  void vcycle_fused(const std::vector<TileList>& fl, int dt, int D, const TileList& tail, size_t tail_smem, T* X, T* F,
                    bool direct, const std::vector<TileList>* rl = nullptr, const std::vector<int>* rfull = nullptr) {
    const double t = sizeof(T);
    float* XS = at<float>(ws, P.w_xs);
    for (int d = 0; d < dt; ++d) {
      if constexpr (sizeof(T) == 4) {
        if (use_reg<T>(rl, d)) {
          const TileList& tl = (*rl)[d];
          go(F_MG_DOWN, (3.5 * t + o.pre_smooth * kfine_extra()) * tl.unk, [&] {
            launch_rdown(G, tiles_at(tl), tl.count, (*rfull)[d], X, XS, F, o.pre_smooth, black_zero(), s);
          });
          continue;
        }
      }
      go(F_MG_DOWN, (3.5 * t + o.pre_smooth * kfine_extra()) * fl[d].unk,
         [&] { launch_mg_down<T>(G, tiles_at(fl[d]), fl[d].count, X, F, o.pre_smooth, o.omega, s); });
    }
    const T* inv = direct ? at<T>(ws, P.w_cinv) : nullptr;
    if (dt == D && !direct &&
        coarsest_smem_bytes(P.kappa_kind, P.strip_coarse_nodes, sizeof(T)) <= 220 * 1024) {
      // the tail is the coarsest grid alone: staged sweeps with precomputed coefficients
      go(F_COARSEST, 4 * t * tail.unk, [&] {
        launch_coarsest_smem<T>(G, tiles_at(tail), tail.count, P.strip_coarse_nodes, X, F, o.coarse_sweeps, o.omega,
                                s);
      });
    } else {
      go(F_MG_TAIL, 3.0 * t * tail.unk, [&] {
        // nd_max sizes the dense-solve buffer, which only direct (subdomain) tails have: it
        // must match the planner's shared-memory size
        launch_mg_tail<T>(G, tiles_at(tail), tail.count, X, F, inv, direct ? P.nd_max : 0, D - dt + 1,
                          o.pre_smooth, o.post_smooth, o.coarse_sweeps, o.omega, dt == 0 ? 1 : 0, tail_smem, s);
      });
    }
    for (int d = dt - 1; d >= 0; --d) {
      if constexpr (sizeof(T) == 4) {
        if (use_reg<T>(rl, d)) {
          const TileList& tl = (*rl)[d];
          go(F_MG_UP, (3.25 * t + o.post_smooth * kfine_extra()) * tl.unk, [&] {
            launch_rup(G, tiles_at(tl), tl.count, (*rfull)[d], XS, X, F, o.post_smooth, red_only(), s);
          });
          continue;
        }
      }
      go(F_MG_UP, (3.25 * t + o.post_smooth * kfine_extra()) * fl[d].unk,
         [&] { launch_mg_up<T>(G, tiles_at(fl[d]), fl[d].count, X, F, o.post_smooth, o.omega, s); });
    }
  }

  // Hybrid V-cycle (opts.fused = 2): one launch per operation on the depths above the tail
  // (large grids, many blocks), then the tail kernel for every coarser grid of the jobs.
  template <typename T>
  void vcycle_hybrid(const std::vector<TileList>& lists, int dt, int D, const TileList& tail, size_t tail_smem, T* X,
                     T* F, bool direct, const std::vector<TileList>* rl = nullptr,
                     const std::vector<int>* rfull = nullptr) {
    const double t = sizeof(T);
    float* XS = at<float>(ws, P.w_xs);
    auto smooth = [&](int d, int color) {
      go(F_SMOOTH, (2 * t + 0.5 * kfine_extra()) * lists[d].unk,
         [&] { launch_smooth<T>(G, tiles_at(lists[d]), lists[d].count, X, F, color, o.omega, s); });
    };
    // the first reg_depths depths: the register-blocked legs (pre-smoothing, residual and
    // restriction in one launch; prolongation and post-smoothing in one), the per-operation
    // kernels below them; both leave the coarse grid's x = 0 and f = P^T r
    auto reg = [&](int d) {
      if constexpr (sizeof(T) == 4) return d < o.reg_depths && rl && (int)rl->size() > d && use_reg<T>(rl, d);
      return false;
    };
    for (int d = 0; d < dt; ++d) {
      if constexpr (sizeof(T) == 4) {
        if (reg(d)) {
          const TileList& tl = (*rl)[d];
          go(F_MG_DOWN, (3.5 * t + o.pre_smooth * kfine_extra()) * tl.unk, [&] {
            launch_rdown(G, tiles_at(tl), tl.count, (*rfull)[d], X, XS, F, o.pre_smooth, black_zero(), s);
          });
          continue;
        }
      }
      for (int k = 0; k < o.pre_smooth; ++k) {
        smooth(d, 0);
        smooth(d, 1);
      }
      go(F_RESTRICT, (10 * t + 4 * kfine_extra()) * lists[d + 1].unk,
         [&] { launch_restrict<T>(G, tiles_at(lists[d + 1]), lists[d + 1].count, X, F, black_zero(), s); });
    }
    const T* inv = direct ? at<T>(ws, P.w_cinv) : nullptr;
    if (dt == D && !direct && coarsest_smem_bytes(P.kappa_kind, P.strip_coarse_nodes, sizeof(T)) <= 220 * 1024) {
      go(F_COARSEST, 4 * t * tail.unk, [&] {
        launch_coarsest_smem<T>(G, tiles_at(tail), tail.count, P.strip_coarse_nodes, X, F, o.coarse_sweeps, o.omega,
                                s);
      });
    } else {
      go(F_MG_TAIL, 3.0 * t * tail.unk, [&] {
        launch_mg_tail<T>(G, tiles_at(tail), tail.count, X, F, inv, direct ? P.nd_max : 0, D - dt + 1, o.pre_smooth,
                          o.post_smooth, o.coarse_sweeps, o.omega, dt == 0 ? 1 : 0, tail_smem, s);
      });
    }
    for (int d = dt - 1; d >= 0; --d) {
      if constexpr (sizeof(T) == 4) {
        if (reg(d)) {
          const TileList& tl = (*rl)[d];
          go(F_MG_UP, (3.25 * t + o.post_smooth * kfine_extra()) * tl.unk, [&] {
            launch_rup(G, tiles_at(tl), tl.count, (*rfull)[d], XS, X, F, o.post_smooth, red_only(), s);
          });
          continue;
        }
      }
      go(F_PROLONG, 2.25 * t * lists[d].unk,
         [&] { launch_prolong<T>(G, tiles_at(lists[d]), lists[d].count, X, red_only(), s); });
      for (int k = 0; k < o.post_smooth; ++k) {
        smooth(d, 1);
        smooth(d, 0);
      }
    }
  }

  // passes of V-cycles with FP64 residual refinement in between (mixed) on one job set
  template <typename T>
  void solve_set(const std::vector<TileList>& lists, const TileList& coarsest, int vcycles, T* X, T* F, double* X64,
                 const double* R, int cmode, const std::vector<TileList>* fl = nullptr, int dt = 0,
                 const TileList* tail = nullptr, size_t tail_smem = 0, bool rmask = false, bool accum_out = true,
                 const std::vector<TileList>* rl = nullptr, const std::vector<int>* rfull = nullptr) {
    const int D = (int)lists.size() - 1;
    const bool fused = o.fused == 1 && fl && tail && dt <= D && o.pre_smooth >= 1 && o.pre_smooth <= 2 &&
                       o.post_smooth >= 1 && o.post_smooth <= 2;
    const bool hybrid = o.fused == 2 && tail && dt <= D;
    const bool mixed = sizeof(T) == 4;
    const double t = sizeof(T);
    const int passes = mixed ? o.refine_passes : 1;
    const int cyc = mixed ? vcycles : vcycles * o.refine_passes;
    const TileList& top = lists[0];
    for (int pass = 0; pass < passes; ++pass) {
      if (pass > 0) {
        go(F_ACCUM, (2 * t + 16) * top.unk, [&] { launch_accumulate<T>(G, tiles_at(top), top.count, X, X64, s); });
        go(F_REFINE, (16 + t + kfine_extra()) * top.unk, [&] {
          if (rmask)  // subdomain j's right-hand side is R on closed G_j only (adjoint solves)
            launch_refine_residual_masked<T>(G, P.glay, tiles_at(top), top.count, F, X64, R, s);
          else
            launch_refine_residual<T>(G, P.glay, tiles_at(top), top.count, F, X64, R, s);
        });
      }
      for (int v = 0; v < cyc; ++v) {
        if (fused)
          vcycle_fused<T>(*fl, dt, D, *tail, tail_smem, X, F, cmode == C_DIRECT, rl, rfull);
        else if (hybrid)
          vcycle_hybrid<T>(lists, dt, D, *tail, tail_smem, X, F, cmode == C_DIRECT, rl, rfull);
        else
          vcycle<T>(lists, coarsest, X, F, cmode);
      }
    }
    if (mixed && accum_out)
      go(F_ACCUM, (2 * t + 16) * top.unk, [&] { launch_accumulate<T>(G, tiles_at(top), top.count, X, X64, s); });
  }

  template <typename T>
  int run(double* lambda_out, double* u_out) {
    const int B = P.B, n = P.n;
    const bool mixed = sizeof(T) == 4;
    const double t = sizeof(T);
    G.grids = at<GridDesc>(ws, P.w_grids);
    G.regions = at<uint8_t>(ws, P.w_regions);
    G.qlabel = at<int16_t>(ws, P.w_qlabel);
    G.cell_in = at<uint8_t>(ws, P.w_cellin);
    G.sub_top = at<int>(ws, P.w_subtop);
    G.tmaps = at<unsigned char>(ws, P.w_tmaps);
    G.status = reinterpret_cast<unsigned long long*>(at<long long>(ws, P.w_stat) + MLEV_STAT_FLAGS);
    G.ncx = P.ncx;
    G.ncy = P.ncy;
    G.m = P.m;
    G.H = P.H;
    G.kap = P.kap_template;
    double* klvl = at<double>(ws, P.w_klvl);
    float* klvl_f = at<float>(ws, P.w_klvl_f);
    float* kcf = at<float>(ws, P.w_kcf);
    G.kap.lvl = klvl;
    G.kap.lvl_f = klvl_f;
    G.kap.coarse = P.kappa_kind == MLEV_KAPPA_PER_COARSE_CELL ? kappa_src : nullptr;
    G.kap.coarse_f = P.kappa_kind == MLEV_KAPPA_PER_COARSE_CELL ? kcf : nullptr;
    (void)cudaGetLastError();  // do not attribute an earlier unrelated failure to this solve
    long long* stat = at<long long>(ws, P.w_stat);
    const int stat_stride = mlev_stat_stride(n);
    cudaMemsetAsync(stat, 0, P.w_stat.bytes, s);
    double* jobnorm = at<double>(ws, P.w_jobnorm);
    count = 0;
    // ---- coefficient on every level, coarse pencil
    if (P.kappa_kind == MLEV_KAPPA_PER_FINE_ELEM) {
      go(F_KAPPA, 20.0 * B * P.lvl_nx(n) * P.lvl_ny(n) * 2,
         [&] { launch_kappa_copy_fine(G.kap, n, B, kappa_src, klvl, klvl_f, s); });
      for (int l = n - 1; l >= P.l1_lc; --l)
        go(F_KAPPA, 44.0 * B * P.lvl_nx(l) * P.lvl_ny(l) * 2,
           [&] { launch_kappa_average(G.kap, l, B, klvl, klvl_f, s); });
    } else if (P.kappa_kind == MLEV_KAPPA_PER_COARSE_CELL) {
      go(F_KAPPA, 12.0 * B * P.ncx * P.ncy, [&] { launch_kappa_to_f((long long)B * P.ncx * P.ncy, kappa_src, kcf, s); });
      for (int l = -1; l >= P.l1_lc; --l)
        go(F_KAPPA, 44.0 * B * P.lvl_nx(l) * P.lvl_ny(l) * 2,
           [&] { launch_kappa_average(G.kap, l, B, klvl, klvl_f, s); });
    }
    double* KH = at<double>(ws, P.w_band);
    double* MH = KH + (size_t)B * P.nhb * (P.bw + 1);
    go(F_BAND, 16.0 * B * P.nhb * (P.bw + 1), [&] { launch_band_setup(G, B, P.nhb, P.bw, KH, MH, s); });
    // coarsest-grid solvers: dense inverses of the subdomain T_H windows (shared by every
    // correction level), staged sweeps for the strip when its T_{h_2} grid fits on chip
    const int sub_cmode = P.sub_direct ? C_DIRECT : C_SWEEPS;
    const int strip_cmode =
        coarsest_smem_bytes(P.kappa_kind, P.strip_coarse_nodes, sizeof(T)) <= 220 * 1024 ? C_SMEM : C_SWEEPS;
    if (P.sub_direct) {
      const TileList& cl = P.lp[n].sub_coarsest;
      T* inv = at<T>(ws, P.w_cinv);
      go(F_COARSEST, 8.0 * cl.count * P.nd_max * P.nd_max,
         [&] { launch_coarse_inverse<T>(G, tiles_at(cl), cl.count, inv, P.nd_max, s); });
    }
    double* ut[2] = {at<double>(ws, P.w_ut[0]), at<double>(ws, P.w_ut[1])};
    double* uin = at<double>(ws, P.w_uin);
    double* r = at<double>(ws, P.w_r);
    double* lam = at<double>(ws, P.w_lam);
    double* c = at<double>(ws, P.w_c);
    double* c0 = at<double>(ws, P.w_c0);
    const size_t ncoef = (size_t)(P.ncx + 1) * (P.ncy + 1);
    auto utL = [&](int l) { return ck_ut ? ck_ut + (size_t)(l - 1) * B * P.glay.bstride : ut[l & 1]; };
    auto cL = [&](int l) { return ck_c ? ck_c + (size_t)l * B * ncoef : c; };
    auto c0L = [&](int l) { return ck_c0 ? ck_c0 + (size_t)l * B : c0; };
    // several eigenpairs: q virtual members per problem (kern_multi.cu)
    const bool multi = P.q > 1;
    SubEigArgs se{};
    if (multi) {
      se.q = P.q;
      se.s = P.msub;
      se.X = at<double>(ws, P.w_mX);
      se.Y = at<double>(ws, P.w_mY);
      se.AY = at<double>(ws, P.w_mAY);
      se.BY = at<double>(ws, P.w_mBY);
      se.theta = at<double>(ws, P.w_mth);
      se.tol = 1e-10;
      se.rtol = 1e-10;
      se.res_slot = -1;
      se.stat = stat;
      se.stat_stride = stat_stride;
    }
    // ---- Algorithm 4.2 step 1: eigenproblem on V_{0h_1}
    if (multi) {
      const int nx1 = P.lvl_nx(1);
      double* K1 = at<double>(ws, P.w_mk1);
      double* M1 = at<double>(ws, P.w_mm1);
      go(F_BAND, 16.0 * P.Breal * P.m_nb1 * (nx1 + 1),
         [&] { launch_band_level(G, P.Breal, P.q, 1, K1, M1, s); });
      SubEigArgs a1 = se;
      a1.nb = P.m_nb1;
      a1.bwk = nx1 - 1;
      a1.bwm = nx1;
      a1.nbord = 0;
      a1.K = K1;
      a1.M = M1;
      a1.kstride = a1.mstride = (long long)P.m_nb1 * (nx1 + 1);
      a1.max_iter = std::max(o.level1_max_iter, 100);
      a1.init_border = 0;
      a1.it_slot = MLEV_STAT_L1_IT;
      a1.res_slot = MLEV_STAT_L1_RES;
      a1.noconv_flag = MLEV_ST_LEVEL1_NOCONV;
      go(F_LEVEL1, 0.0, [&] { launch_sub_eig(G, a1, P.Breal, s); });
      go(F_LEVEL1, 0.0, [&] {
        launch_level1_multi_out(G, P.glay, P.Breal, P.q, P.msub, a1.X, a1.theta, utL(1), lam, n + 1, cL(1), c0L(1), s);
      });
    } else {
      Level1Args a{};
      a.B = B;
      a.grid_begin = P.l1_grid_begin;
      a.nlev = P.l1_nlev;
      a.vec = at<double>(ws, P.w_l1vec);
      a.vstride = P.w_l1vec.bytes / 8 / 10 / B;
      a.xpool = at<void>(ws, P.w_l1pool[0]);
      a.fpool = at<void>(ws, P.w_l1pool[1]);
      a.pre = o.pre_smooth;
      a.post = o.post_smooth;
      a.coarse_sweeps = std::max(4, o.coarse_sweeps / 4);  // level-1 coarsest grid: a few nodes
      a.omega = o.omega;
      a.max_iter = o.level1_max_iter;
      a.tol = o.level1_tol;
      a.ut1 = utL(1);
      a.lam = lam;
      a.lam_stride = n + 1;
      a.c = cL(1);
      a.c0 = c0L(1);
      a.stat = stat;
      a.stat_stride = stat_stride;
      long long nn0 = 0, tot = 0;
      for (int k = 0; k < P.l1_nlev; ++k) {
        const GridDesc& gk = P.grids[P.l1_grid_begin + k];
        const long long nk = (long long)(gk.nx + 1) * (gk.ny + 1);
        if (k == 0) nn0 = nk;
        tot += (nk + 1) & ~1LL;
      }
      const size_t l1smem = level1_smem_bytes(nn0, tot, sizeof(T));
      if (l1smem <= (size_t)kL1SmemMax)
        go(F_LEVEL1, 0.0, [&] { launch_level1_sm<T>(G, P.glay, a, l1smem, s); });
      else
        go(F_LEVEL1, 0.0, [&] { launch_level1<T>(G, P.glay, a, s); });
    }
    T* X = at<T>(ws, P.w_x);
    T* F = at<T>(ws, P.w_f);
    double* X64 = mixed ? at<double>(ws, P.w_x64) : nullptr;
    double* partials = at<double>(ws, P.w_aug);
    // ---- Algorithm 4.2 step 3: Correction on levels 2..n
    for (int L = 2; L <= n; ++L) {
      const LevelPlan& lp = P.lp[L];
      const double nfree = (double)lp.n_free * B;
      G.sub_top = at<int>(ws, P.w_subtop) + lp.sub_top_off;
      LevelArgs a{};
      a.L = L;
      a.B = B;
      {
        const double h = P.H / (double)(1 << L);  // exact: the kernels' h_L
        a.m12 = h * h / 12.0;
      }
      a.ut_prev = utL(L - 1);
      if (multi && L >= 3) {
        // u_{i,h_{L-1}} = sum_j D_ij u~_j + P_H c_i: the u~ combination into the buffer that
        // level L's glue fills afterwards (only the embedding reads ut_prev before that)
        double* comb = ut[L & 1];
        const double* Dm = at<double>(ws, P.w_mD);
        const double* src = utL(L - 1);
        go(F_INTERP, 16.0 * B * P.lvl_nx(L - 1) * P.lvl_ny(L - 1),
           [&] { launch_combine(P.glay, L - 1, P.Breal, P.q, Dm, src, comb, s); });
        a.ut_prev = comb;
      }
      a.ut = utL(L);
      a.uin = uin;
      a.r = r;
      a.c = cL(L - 1);
      a.c0 = c0L(L - 1);
      a.lam = lam;
      a.lam_stride = n + 1;
      RRArgs rr{};
      rr.B = B;
      rr.L = L;
      rr.n = n;
      rr.nhb = P.nhb;
      rr.bw = P.bw;
      rr.KH = KH;
      rr.MH = MH;
      rr.chol = at<double>(ws, P.w_chol);
      rr.partials = partials;
      rr.lam = lam;
      rr.c = cL(L);
      rr.c0 = c0L(L);
      rr.c_prev = cL(L - 1);
      rr.c0_prev = c0L(L - 1);
      rr.stat = stat;
      rr.stat_stride = stat_stride;
      rr.max_iter = o.rr_max_iter;
      rr.mixed = (mixed && rr_mixed_supported(P.nhb, P.bw)) ? 1 : 0;
      // row-blocked solves: one warp holds a grid row of the coarse system (<= 32 nodes)
      rr.blocked = rr.mixed && P.bw - 1 <= 32 && rr_mixed_smem_bytes(P.nhb, P.bw, 1) <= (size_t)kRRSmemMax ? 1 : 0;
      rr.smem = (rr.mixed ? rr_mixed_smem_bytes(P.nhb, P.bw, rr.blocked) : rr_smem_bytes(P.nhb, P.bw)) <=
                (size_t)kRRSmemMax;
      // the Rayleigh-Ritz factors of this level are prepared by the inner-product kernel
      // (they need only K_H, M_H and the eigenvalues of the earlier levels)
      rr.pre = at<unsigned char>(ws, P.w_rrpre);
      rr.pre_stride = (long long)mlev_rr_prefactor_stride(P.nhb, P.bw);
      // only where the inner-product kernel, every block then holding the factor's shared
      // memory, still runs in one wave (a batch of many problems would lose occupancy there)
      const size_t pre_smem = rr_prefactor_smem(P.nhb, P.bw);
      const long long aug_cells = (long long)B * P.ncx * P.ncy;
      const long long aug_blocks = L <= 5 ? B + (aug_cells + 7) / 8 : aug_cells + B;  // warp or block per cell
      // (per block: the factor's dynamic memory, the kernel's 22.6 KB of static staging and the
      // 1 KB the runtime reserves)
      const long long aug_slots = (long long)ctx->sm_count * (long long)(ctx->smem_per_sm / (pre_smem + 24 * 1024));
      rr.use_pre = rr.blocked && rr.smem && L >= 3 && P.bw - 1 <= 16 && P.w_rrpre.bytes > 0 &&
                           pre_smem <= (size_t)kRRSmemMax && aug_blocks <= aug_slots ? 1 : 0;
      const RRPrefactor pf{KH, MH, P.nhb, P.bw, rr.pre, rr.pre_stride};
      go(F_INTERP, 10.0 * nfree, [&] { launch_interp(G, P.glay, a, s); });
      go(F_RHS, (16.0 + kfine_extra()) * nfree, [&] { launch_rhs(G, P.glay, a, s); });
      // multigrid pools of this level start at zero: nodes that are not unknowns must read
      // as 0 (the fused kernels skip tiles without unknowns)
      cudaMemsetAsync(X, 0, (size_t)lp.pool_elems * sizeof(T), s);
      // step 1: auxiliary problems on every Omega_j of every batch member
      const TileList& top = lp.sub[0];
      // with one pass the FP64 accumulator would only be the FP32 solution widened: glue and
      // the strip update read the FP32 pool directly (same values) unless residuals are checked,
      // and the accumulator is neither zeroed nor written
      const bool direct32 = mixed && o.refine_passes == 1 && !o.check_residuals;
      double* X64z = direct32 ? nullptr : X64;
      go(F_GATHER, (8 + t + (X64z ? 8 : 0)) * top.unk,
         [&] { launch_gather<T>(G, P.glay, tiles_at(top), top.count, X, F, X64z, r, s); });
      const float* E32 = direct32 ? reinterpret_cast<const float*>(X) : nullptr;
      solve_set<T>(lp.sub, lp.sub_coarsest, o.vcycles, X, F, X64, r, sub_cmode, &lp.sub_f, lp.sub_dt, &lp.sub_tail,
                   lp.sub_tail_smem, false, !direct32, &lp.sub_r, &lp.sub_r_full);
      const double* E = mixed ? X64 : reinterpret_cast<const double*>(X);
      if (o.check_residuals) {
        cudaMemsetAsync(jobnorm, 0, P.w_jobnorm.bytes, s);
        go(F_RESNORM, 16.0 * top.unk,
           [&] { launch_job_resnorm(G, P.glay, tiles_at(top), top.count, E, mixed ? 1 : 0, r, jobnorm, s); });
        go(F_RESNORM, 0.0,
           [&] { launch_resnorm_finalize(jobnorm, B, P.m, 1, stat, stat_stride, MLEV_STAT_LOC_RES(n) + L, s); });
      }
      // step 2: glue, then the G_{m+1} problem
      go(F_GLUE, 24.0 * nfree, [&] { launch_glue(G, P.glay, a, E, mixed ? 1 : 0, E32, s); });
      const TileList& stop = lp.strip[0];
      if (stop.count) {
        go(F_STRIP_RHS, (32.0 + 2 * t + (X64z ? 8 : 0) + kfine_extra()) * stop.unk,
           [&] { launch_strip_rhs<T>(G, P.glay, a, tiles_at(stop), stop.count, X, F, X64z, s); });
        solve_set<T>(lp.strip, lp.strip_coarsest, o.strip_vcycles, X, F, X64, r, strip_cmode, &lp.strip_f,
                     lp.strip_dt, &lp.strip_tail, lp.strip_tail_smem, false, !direct32, &lp.strip_r, &lp.strip_r_full);
        if (o.check_residuals) {
          cudaMemsetAsync(jobnorm, 0, P.w_jobnorm.bytes, s);
          go(F_RESNORM, 16.0 * stop.unk,
             [&] { launch_job_resnorm(G, P.glay, tiles_at(stop), stop.count, E, mixed ? 1 : 0, r, jobnorm, s); });
          go(F_RESNORM, 0.0,
             [&] { launch_resnorm_finalize(jobnorm, B, P.m, 0, stat, stat_stride, MLEV_STAT_STRIP_RES(n) + L, s); });
        }
        go(F_STRIP_UPD, 24.0 * stop.unk,
           [&] { launch_strip_update(G, P.glay, a, tiles_at(stop), stop.count, E, mixed ? 1 : 0, E32, s); });
      }
      // step 3: Rayleigh-Ritz on V_{0H} + span{u~}
      if (multi) rr.use_pre = 0;
      go(F_AUG, (8.0 + kfine_extra()) * nfree,
         [&] { launch_aug(G, P.glay, a, partials, rr.use_pre ? &pf : nullptr, s); });
      if (multi) {  // ... + span{u~_1 .. u~_q}: Gram matrices, bordered pencil, subspace iteration
        double* cross = at<double>(ws, P.w_mcross);
        SubEigArgs ar = se;
        ar.nb = P.nhb;
        ar.bwk = P.bw - 1;
        ar.bwm = P.bw;
        ar.nbord = P.q;
        ar.K = KH;
        ar.M = MH;
        ar.kstride = ar.mstride = (long long)P.q * P.nhb * (P.bw + 1);
        ar.Ga = at<double>(ws, P.w_mGa);
        ar.Gb = at<double>(ws, P.w_mGb);
        ar.Aq = at<double>(ws, P.w_mAq);
        ar.Bq = at<double>(ws, P.w_mBq);
        ar.Z = at<double>(ws, P.w_mZ);
        ar.max_iter = std::max(o.rr_max_iter, 50);
        ar.init_border = 1;
        ar.it_slot = MLEV_STAT_RR_IT + L;
        ar.noconv_flag = MLEV_ST_RR_NOCONV;
        const int npq = P.q * (P.q + 1) / 2;
        go(F_AUG, 16.0 * nfree * npq / P.q, [&] { launch_cross_gram(G, P.glay, L, P.Breal, P.q, utL(L), cross, s); });
        go(F_RR, 0.0, [&] {
          launch_border_prep(G, P.Breal, P.q, partials, cross, at<double>(ws, P.w_mGa), at<double>(ws, P.w_mGb),
                             at<double>(ws, P.w_mAq), at<double>(ws, P.w_mBq), s);
        });
        go(F_RR, 0.0, [&] { launch_sub_eig(G, ar, P.Breal, s); });
        go(F_RR, 0.0, [&] {
          launch_rr_multi_out(G, P.Breal, P.q, P.msub, P.nhb, P.bw, L, n + 1, ar.X, ar.theta, MH, ar.mstride, ar.Gb,
                              cL(L), c0L(L), at<double>(ws, P.w_mD), lam, s);
        });
      } else {
        go(F_RR, 0.0, [&] { launch_rr(G, rr, s); });
      }
    }
    go(F_OUT, 16.0 * B, [&] { launch_lambda_out(B, n, lam, lambda_out, s); });
    if (u_out) {
      const double* ufield = utL(n);
      if (multi) {  // u_{i,h_n} = sum_j D_ij u~_j + P_H c_i
        double* comb = ut[(n + 1) & 1];
        const double* Dm = at<double>(ws, P.w_mD);
        go(F_OUT, 16.0 * B * P.lvl_nx(n) * P.lvl_ny(n),
           [&] { launch_combine(P.glay, n, P.Breal, P.q, Dm, utL(n), comb, s); });
        ufield = comb;
      }
      go(F_OUT, 16.0 * B * (P.lvl_nx(n) + 1) * (P.lvl_ny(n) + 1),
         [&] { launch_output_u(G, P.glay, n, B, ufield, cL(n), c0L(n), u_out, s); });
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    return MLEV_OK;
  }

  // Forward pass with level checkpoints, then the reverse sweep of Algorithm 4.2 for
  // dlambda_{h_n}/dkappa (kernels and the derivation: kern_adj.cu).
  template <typename T>
  int run_grad(const double* dl, int layout, double* dkappa, double* lambda_out) {
    const int B = P.B, n = P.n;
    const bool mixed = sizeof(T) == 4;
    const double t = sizeof(T);
    const int ncoef = (P.ncx + 1) * (P.ncy + 1);
    const size_t gfield = (size_t)B * P.glay.bstride;
    ck_ut = at<double>(ws, P.g_ck_ut);
    ck_c = at<double>(ws, P.g_ck_c);
    ck_c0 = at<double>(ws, P.g_ck_c0);
    int rc = run<T>(lambda_out ? lambda_out : at<double>(ws, P.w_out_lam), nullptr);
    if (rc) return rc;
    double* lam = at<double>(ws, P.w_lam);
    double* lambar = at<double>(ws, P.g_lambar);
    double* ubar[2] = {at<double>(ws, P.g_ubar[0]), at<double>(ws, P.g_ubar[1])};
    double* utbar = at<double>(ws, P.g_utbar);
    double* sbar = at<double>(ws, P.g_sbar);
    double* rbar = at<double>(ws, P.g_rbar);
    double* tbuf = at<double>(ws, P.g_tbuf);
    double* glb = at<double>(ws, P.g_gl);
    double* coef = at<double>(ws, P.g_coef);
    double* part2 = at<double>(ws, P.g_part2);
    double* lbpart = at<double>(ws, P.g_lbpart);
    double* uin = at<double>(ws, P.w_uin);
    double* r = at<double>(ws, P.w_r);
    double* partials = at<double>(ws, P.w_aug);
    double* KH = at<double>(ws, P.w_band);
    double* MH = KH + (size_t)B * P.nhb * (P.bw + 1);
    long long* stat = at<long long>(ws, P.w_stat);
    const int stat_stride = mlev_stat_stride(n);
    const int cstride = 3 * ncoef + kAdjScal;
    T* X = at<T>(ws, P.w_x);
    T* F = at<T>(ws, P.w_f);
    double* X64 = mixed ? at<double>(ws, P.w_x64) : nullptr;
    const double* E = mixed ? X64 : reinterpret_cast<const double*>(X);
    const int use64 = mixed ? 1 : 0;
    const int sub_cmode = P.sub_direct ? C_DIRECT : C_SWEEPS;
    const int strip_cmode =
        coarsest_smem_bytes(P.kappa_kind, P.strip_coarse_nodes, sizeof(T)) <= 220 * 1024 ? C_SMEM : C_SWEEPS;
    cudaMemsetAsync(glb, 0, P.g_gl.bytes, s);
    cudaMemsetAsync(ubar[n & 1], 0, gfield * 8, s);
    go(F_ADJ_FIELD, 0.0, [&] { launch_lambar_init(B, n, dl, lambar, s); });
    for (int L = n; L >= 2; --L) {
      const int k = L - 1;
      const LevelPlan& lp = P.lp[L];
      const double nfree = (double)lp.n_free * B;
      G.sub_top = at<int>(ws, P.w_subtop) + lp.sub_top_off;
      double* gL = glb + P.gl_off[L];
      double* ubL = ubar[L & 1];
      double* utl = ck_ut + (size_t)(L - 1) * gfield;
      LevelArgs a{};
      a.L = L;
      a.B = B;
      {
        const double h = P.H / (double)(1 << L);  // exact: the kernels' h_L
        a.m12 = h * h / 12.0;
      }
      a.ut_prev = ck_ut + (size_t)(k - 1) * gfield;
      a.ut = utl;
      a.uin = uin;
      a.r = r;
      a.c = ck_c + (size_t)k * B * ncoef;
      a.c0 = ck_c0 + (size_t)k * B;
      a.lam = lam;
      a.lam_stride = n + 1;
      // u_in and r of the forward level (cheap to recompute), inner products of u~_L
      go(F_INTERP, 10.0 * nfree, [&] { launch_interp(G, P.glay, a, s); });
      go(F_RHS, (16.0 + kfine_extra()) * nfree, [&] { launch_rhs(G, P.glay, a, s); });
      go(F_AUG, (8.0 + kfine_extra()) * nfree, [&] { launch_aug(G, P.glay, a, partials, nullptr, s); });
      // Rayleigh-Ritz adjoint
      go(F_ADJ_FIELD, 16.0 * nfree, [&] { launch_cbar(G, P.glay, L, B, utl, ubL, part2, s); });
      RRAdjArgs ra{};
      ra.B = B;
      ra.L = L;
      ra.n = n;
      ra.nhb = P.nhb;
      ra.bw = P.bw;
      ra.KH = KH;
      ra.MH = MH;
      ra.scratch = at<double>(ws, P.g_rrscr);
      ra.smem = rr_adj_smem_bytes(P.nhb, P.bw) <= (size_t)kRRSmemMax;
      ra.partials = partials;
      ra.part2 = part2;
      ra.lam = lam;
      ra.lambar = lambar;
      ra.c = ck_c + (size_t)L * B * ncoef;
      ra.c0 = ck_c0 + (size_t)L * B;
      ra.coef = coef;
      ra.cstride = cstride;
      ra.stat = stat;
      ra.stat_stride = stat_stride;
      go(F_ADJ_RR, 0.0, [&] { launch_rr_adj(G, ra, s); });
      go(F_ADJ_FIELD, 32.0 * nfree, [&] { launch_adj_ut(G, P.glay, L, B, utl, ubL, coef, cstride, utbar, s); });
      const AugField fu{ck_c + (size_t)L * B * ncoef, ncoef, ck_c0 + (size_t)L * B, 1, utl};
      const AugField fz{coef, cstride, coef + 3 * ncoef + ADJ_ZU, cstride, utl};
      go(F_ADJ_GRAD, 24.0 * nfree, [&] { launch_grad_aug(G, P.glay, L, B, fu, fz, lambar + L, n + 1, -1.0, gL, s); });
      // G_{m+1} adjoint: K_SS sbar = utbar on the strip
      cudaMemsetAsync(sbar, 0, gfield * 8, s);
      const TileList& stop = lp.strip[0];
      if (stop.count) {
        cudaMemsetAsync(X, 0, (size_t)lp.pool_elems * sizeof(T), s);
        go(F_GATHER, (8 + t + (mixed ? 8 : 0)) * stop.unk,
           [&] { launch_gather<T>(G, P.glay, tiles_at(stop), stop.count, X, F, X64, utbar, s); });
        solve_set<T>(lp.strip, lp.strip_coarsest, o.strip_vcycles, X, F, X64, utbar, strip_cmode, &lp.strip_f,
                     lp.strip_dt, &lp.strip_tail, lp.strip_tail_smem, false, true, &lp.strip_r, &lp.strip_r_full);
        LevelArgs as = a;
        as.ut = sbar;
        go(F_STRIP_UPD, 24.0 * stop.unk,
           [&] { launch_strip_update(G, P.glay, as, tiles_at(stop), stop.count, E, use64, nullptr, s); });
        go(F_ADJ_FIELD, 24.0 * nfree, [&] { launch_strip_adj_post(G, P.glay, L, B, utbar, sbar, s); });
        go(F_ADJ_GRAD, 16.0 * nfree, [&] { launch_grad_pair(G, P.glay, L, B, -1.0, sbar, utl, gL, s); });
      }
      // local adjoints t_j = A_j^{-1} (utbar on closed G_j), kept aside
      const TileList& top = lp.sub[0];
      cudaMemsetAsync(X, 0, (size_t)lp.pool_elems * sizeof(T), s);
      go(F_GATHER, (8 + 2 * t + (mixed ? 8 : 0)) * top.unk,
         [&] { launch_gather_masked<T>(G, P.glay, tiles_at(top), top.count, X, F, X64, utbar, s); });
      solve_set<T>(lp.sub, lp.sub_coarsest, o.vcycles, X, F, X64, utbar, sub_cmode, &lp.sub_f, lp.sub_dt,
                   &lp.sub_tail, lp.sub_tail_smem, true, true, &lp.sub_r, &lp.sub_r_full);
      const size_t ebytes = (size_t)(mixed ? lp.pool64_elems : lp.pool_elems) * 8;
      cudaMemcpyAsync(tbuf, E, ebytes, cudaMemcpyDeviceToDevice, s);
      // the forward local solutions e^j, recomputed
      cudaMemsetAsync(X, 0, (size_t)lp.pool_elems * sizeof(T), s);
      go(F_GATHER, (8 + t + (mixed ? 8 : 0)) * top.unk,
         [&] { launch_gather<T>(G, P.glay, tiles_at(top), top.count, X, F, X64, r, s); });
      solve_set<T>(lp.sub, lp.sub_coarsest, o.vcycles, X, F, X64, r, sub_cmode, &lp.sub_f, lp.sub_dt, &lp.sub_tail,
                   lp.sub_tail_smem, false, true, &lp.sub_r, &lp.sub_r_full);
      go(F_ADJ_GRAD, 32.0 * top.unk, [&] { launch_grad_local(G, P.glay, L, B, tbuf, E, use64, uin, gL, s); });
      go(F_ADJ_FIELD, 8.0 * top.unk + 8.0 * nfree, [&] { launch_rbar(G, P.glay, L, B, tbuf, use64, rbar, s); });
      const int nblk = adj_uin_blocks(P.glay, L);
      go(F_ADJ_FIELD, 40.0 * nfree, [&] {
        launch_adj_uin(G, P.glay, L, B, utbar, sbar, rbar, uin, lam, n + 1, lbpart, P.adj_nblk, s);
      });
      go(F_ADJ_FIELD, 8.0 * nblk * B,
         [&] { launch_lambar_finalize(B, nblk, P.adj_nblk, lbpart, lambar, n + 1, k, s); });
      go(F_ADJ_FIELD, 16.0 * nfree, [&] { launch_restrict_adj(G, P.glay, k, B, utbar, ubar[k & 1], s); });
    }
    // level 1: eigenvector adjoint, then its element terms
    {
      Level1AdjArgs la{};
      la.B = B;
      la.grid_begin = P.l1_grid_begin;
      la.nlev = P.l1_nlev;
      la.vec = at<double>(ws, P.w_l1vec);
      la.vstride = P.w_l1vec.bytes / 8 / 10 / B;
      la.xpool = at<void>(ws, P.w_l1pool[0]);
      la.fpool = at<void>(ws, P.w_l1pool[1]);
      la.pre = o.pre_smooth;
      la.post = o.post_smooth;
      la.coarse_sweeps = std::max(4, o.coarse_sweeps / 4);
      la.omega = o.omega;
      la.max_iter = 4 * o.level1_max_iter;
      la.tol = 1e-11;
      la.ut1 = ck_ut;
      la.ubar1 = ubar[1];
      la.lam = lam;
      la.lam_stride = n + 1;
      la.zout = sbar;
      la.stat = stat;
      la.stat_stride = stat_stride;
      go(F_ADJ_LEVEL1, 0.0, [&] { launch_level1_adj<T>(G, P.glay, la, s); });
      const AugField f1{nullptr, 0, nullptr, 0, ck_ut}, f2{nullptr, 0, nullptr, 0, sbar};
      go(F_ADJ_GRAD, 24.0 * B * P.lvl_nx(1) * P.lvl_ny(1),
         [&] { launch_grad_aug(G, P.glay, 1, B, f1, f2, lambar + 1, n + 1, -1.0, glb + P.gl_off[1], s); });
    }
    GradLevels gv{};
    for (int l = 1; l <= n; ++l) gv.off[l] = P.gl_off[l];
    go(F_ADJ_GRAD, 16.0 * B * P.lvl_nx(n) * P.lvl_ny(n) * 2,
       [&] { launch_grad_spread(G, P.glay, n, B, gv, glb, layout, dkappa, s); });
    ck_ut = ck_c = ck_c0 = nullptr;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch (adjoint)");
    return MLEV_OK;
  }
};

int ensure_plan(mlev_ctx* ctx, const mlev_opts* o) {
  if (ctx->built_version == ctx->version && ctx->built_precision == o->precision &&
      ctx->built_tail_nodes == o->tail_nodes)
    return MLEV_OK;
  if (fault_armed("plan_alloc")) throw std::bad_alloc();
  int rc = map_plan_error(ctx, ctx->plan.build(*o));
  if (rc) return rc;
  ctx->built_version = ctx->version;
  ctx->built_precision = o->precision;
  ctx->built_tail_nodes = o->tail_nodes;
  ctx->plan_gen++;
  return MLEV_OK;
}

int prepare(mlev_ctx* ctx, const mlev_opts* o, void* ws, size_t ws_bytes) {
  if (!ctx) return MLEV_EINVAL;
  if (ctx->device < 0) return fail(ctx, MLEV_ESTATE, "planning-only context (device -1) cannot solve");
  if (!opts_valid(o)) return fail(ctx, MLEV_EINVAL, "invalid options");
  int rc = ensure_plan(ctx, o);
  if (rc) return rc;
  ctx->io_h2d = ctx->io_d2h = 0;
  if (!ws || ((uintptr_t)ws & 255)) return fail(ctx, MLEV_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < ctx->plan.ws_bytes)
    return fail(ctx, MLEV_ENOMEM, "workspace too small: need " + std::to_string(ctx->plan.ws_bytes) + " bytes");
  return MLEV_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up through the runtime (the library does
// not link libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor maps of the grids read by the fused kernels: boxes over the x and f pools of the
// grid (pitched 2-D arrays of (nx+1) x (ny+1) nodes); out-of-range boxes read zeros.
std::string encode_tensor_maps(const Plan& P, void* ws, char* host) {
  if (!P.n_tmap_grids) return "";
  auto enc = tensor_map_encoder();
  if (!enc) return "cuTensorMapEncodeTiled is not available from the driver";
  const CUtensorMapDataType dt = P.tsize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host + P.w_tmaps.off);
  char* xbase = static_cast<char*>(ws) + P.w_x.off;
  char* fbase = static_cast<char*>(ws) + P.w_f.off;
  for (const GridDesc& g : P.grids) {
    if (g.tmap < 0) continue;
    const cuuint64_t dims[2] = {(cuuint64_t)g.nx + 1, (cuuint64_t)g.ny + 1};
    const cuuint64_t strides[1] = {(cuuint64_t)g.pitch * P.tsize};
    const cuuint32_t fbox[2] = {MLEV_TMA_FBW, MLEV_TMA_FBH}, cbox[2] = {MLEV_TMA_CBW, MLEV_TMA_CBH};
    const cuuint32_t es[2] = {1, 1};
    void* xa = xbase + g.off * P.tsize;
    void* fa = fbase + g.off * P.tsize;
    CUresult r0 = enc(&maps[g.tmap + 0], dt, 2, xa, dims, strides, fbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r1 = enc(&maps[g.tmap + 1], dt, 2, fa, dims, strides, fbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(&maps[g.tmap + 2], dt, 2, xa, dims, strides, cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r0 != CUDA_SUCCESS || r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
      return "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r0) + "/" + std::to_string((int)r1) + "/" +
             std::to_string((int)r2) + ")";
  }
  return "";
}

int upload_tables(mlev_ctx* ctx, void* ws, cudaStream_t s, bool force) {
  Plan& P = ctx->plan;
  const long long key = ctx->plan_gen;
  if (!force && ctx->uploaded_ws == ws && ctx->uploaded_version == key) return MLEV_OK;
  std::vector<char> host(P.tables_bytes, 0);
  auto put = [&](const Span& sp, const void* src, size_t bytes) {
    if (bytes) std::memcpy(host.data() + sp.off, src, bytes);
  };
  put(P.w_grids, P.grids.data(), P.grids.size() * sizeof(GridDesc));
  put(P.w_tiles, P.tiles.data(), P.tiles.size() * sizeof(Tile));
  put(P.w_regions, P.regions.data(), P.regions.size());
  put(P.w_qlabel, P.qlabel.data(), P.qlabel.size() * sizeof(int16_t));
  put(P.w_cellin, P.cell_in.data(), P.cell_in.size());
  put(P.w_subtop, P.sub_top.data(), P.sub_top.size() * sizeof(int));
  std::string terr = encode_tensor_maps(P, ws, host.data());
  if (!terr.empty()) return fail(ctx, MLEV_ECUDA, terr);
  if (fault_armed("h2d_copy")) return cuda_fail(ctx, cudaErrorInvalidValue, "plan table copy (injected fault)");
  CK(cudaMemcpyAsync(ws, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  ctx->io_h2d += (long long)host.size();
  if (!P.kappa_on_device && !P.kappa_host.empty()) {
    const double* ksrc = P.kappa_host.data();
    std::vector<double> krep;
    if (P.q > 1) {  // one copy per virtual member b q + i
      const size_t per = P.kappa_host.size() / (size_t)P.Breal;
      krep.resize(per * (size_t)P.B);
      for (int b = 0; b < P.Breal; ++b)
        for (int i = 0; i < P.q; ++i)
          std::memcpy(krep.data() + ((size_t)b * P.q + i) * per, P.kappa_host.data() + (size_t)b * per, per * 8);
      ksrc = krep.data();
    }
    std::vector<double> knan;
    if (fault_armed("kappa_nan")) {  // first positive value (a cell or triangle of Omega) -> NaN
      knan.assign(ksrc, ksrc + (P.kappa_host.size() / (size_t)P.Breal) * (size_t)P.B);
      for (double& v : knan)
        if (v > 0) {
          v = std::nan("");
          break;
        }
      ksrc = knan.data();
    }
    const size_t kbytes = (P.kappa_host.size() / (size_t)P.Breal) * (size_t)P.B * 8;
    CK(cudaMemcpyAsync(at<char>(ws, P.w_kstage), ksrc, kbytes, cudaMemcpyHostToDevice, s));
    ctx->io_h2d += (long long)kbytes;
  }
  CK(cudaStreamSynchronize(s));
  ctx->uploaded_ws = ws;
  ctx->uploaded_version = key;
  return MLEV_OK;
}

int fill_report(mlev_ctx* ctx, void* ws, cudaStream_t s, mlev_report* rep) {
  const Plan& P = ctx->plan;
  CK(cudaStreamSynchronize(s));
  const int n = P.n, B = P.B, stride = mlev_stat_stride(n);
  std::vector<long long> st((size_t)B * stride);
  std::vector<double> lam((size_t)B * (n + 1));
  CK(cudaMemcpy(st.data(), at<char>(ws, P.w_stat), st.size() * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(lam.data(), at<char>(ws, P.w_lam), lam.size() * 8, cudaMemcpyDeviceToHost));
  std::memset(rep, 0, sizeof(*rep));
  rep->levels = n;
  rep->batch = B;
  for (int k = 1; k <= n; ++k) rep->lambda[k] = lam[k];
  int flags = 0;
  for (int b = 0; b < B; ++b) {
    const long long* sb = st.data() + (size_t)b * stride;
    auto as_double = [](long long v) {
      double d;
      std::memcpy(&d, &v, 8);
      return d;
    };
    rep->level1_iters = std::max(rep->level1_iters, (int)sb[MLEV_STAT_L1_IT]);
    rep->level1_residual = std::max(rep->level1_residual, as_double(sb[MLEV_STAT_L1_RES]));
    flags |= (int)sb[MLEV_STAT_FLAGS];
    for (int k = 2; k <= n; ++k) {
      rep->rr_iters[k] = std::max(rep->rr_iters[k], (int)sb[MLEV_STAT_RR_IT + k]);
      rep->local_residual[k] = std::max(rep->local_residual[k], as_double(sb[MLEV_STAT_LOC_RES(n) + k]));
      rep->strip_residual[k] = std::max(rep->strip_residual[k], as_double(sb[MLEV_STAT_STRIP_RES(n) + k]));
    }
  }
  rep->status_flags = flags;
  rep->n_fine = P.n_fine;
  rep->n_local_fine = P.lp[n].n_local;
  rep->n_strip_fine = P.lp[n].n_strip;
  rep->n_coarse = P.n_coarse;
  rep->kernel_launches = ctx->launches;
  rep->h2d_bytes = ctx->io_h2d;
  rep->d2h_bytes = ctx->io_d2h;
  if (flags & MLEV_ST_TIMEOUT)
    return fail(ctx, MLEV_ETIMEOUT, "a bounded device-side wait gave up (status flags " + std::to_string(flags) + ")");
  if (flags & (MLEV_ST_LEVEL1_NOCONV | MLEV_ST_RR_NOCONV | MLEV_ST_ADJ_NOCONV))
    return fail(ctx, MLEV_ENOCONV, "an iteration reached its cap (status flags " + std::to_string(flags) + ")");
  if (flags & MLEV_ST_NONFINITE)
    return fail(ctx, MLEV_ENOCONV, "non-finite value in the solve (status flags " + std::to_string(flags) + ")");
  if (flags) return fail(ctx, MLEV_ENOCONV, "numerical breakdown (status flags " + std::to_string(flags) + ")");
  return MLEV_OK;
}

int solve_impl(mlev_ctx* ctx, const mlev_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
               const double* kappa_src, double* lambda_out, double* u_out) {
  const Plan& P = ctx->plan;
  Launcher ln{ctx, P, *o, ws, s};
  ln.kappa_src = kappa_src;
  int rc;
  if (o->profile) {
    std::vector<ProfRec> recs;
    ln.profiling = true;
    ln.recs = &recs;
    ln.pool = &ctx->ev_pool;
    rc = o->precision == MLEV_PREC_FP64 ? ln.run<double>(lambda_out, u_out) : ln.run<float>(lambda_out, u_out);
    ctx->launches = ln.count;
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    ctx->prof.assign(F_COUNT, ProfRecHost());
    for (const ProfRec& r : recs) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      ctx->prof[r.fam].launches++;
      ctx->prof[r.fam].ms += ms;
      ctx->prof[r.fam].bytes += r.bytes;
    }
    ctx->prof_valid = true;
    return MLEV_OK;
  }
  if (o->use_graph) {
    char key[256];
    snprintf(key, sizeof key, "%p/%p/%p/%p/%p/%lld/", ws, (void*)s, (void*)lambda_out, (void*)u_out,
             (const void*)kappa_src, ctx->version);
    const std::string k = std::string(key) + opts_key(o);
    if (!ctx->gexec || ctx->graph_key != k) {
      if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
      }
      if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
      cudaGraph_t graph;
      Launcher cap{ctx, P, *o, ws, ctx->capture_stream};
      cap.kappa_src = kappa_src;
      CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
      rc = o->precision == MLEV_PREC_FP64 ? cap.run<double>(lambda_out, u_out) : cap.run<float>(lambda_out, u_out);
      cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
      ln.count = cap.count;
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
      ctx->graph_key = k;
      ctx->graph_launches = ln.count;
    }
    CK(cudaGraphLaunch(ctx->gexec, s));
    ctx->launches = ctx->graph_launches;
    return MLEV_OK;
  }
  rc = o->precision == MLEV_PREC_FP64 ? ln.run<double>(lambda_out, u_out) : ln.run<float>(lambda_out, u_out);
  ctx->launches = ln.count;
  return rc;
}

constexpr double kGradLevel1Tol = 1e-10;

int grad_impl(mlev_ctx* ctx, const mlev_opts* o, void* ws, cudaStream_t s, const double* kappa_src,
              const double* dl, int layout, double* dkappa, double* lambda_out) {
  const Plan& P = ctx->plan;
  // the reverse sweep differentiates an exact level-1 eigenpair (its projected adjoint solve
  // needs u_{h_1} to satisfy the level-1 pencil), so the forward pass solves level 1 to at
  // least kGradLevel1Tol whatever the caller's schedule asks
  mlev_opts og = *o;
  og.level1_tol = std::min(og.level1_tol, kGradLevel1Tol);
  Launcher ln{ctx, P, og, ws, s};
  ln.kappa_src = kappa_src;
  std::vector<ProfRec> recs;
  if (o->profile) {
    ln.profiling = true;
    ln.recs = &recs;
    ln.pool = &ctx->ev_pool;
  }
  int rc = o->precision == MLEV_PREC_FP64 ? ln.run_grad<double>(dl, layout, dkappa, lambda_out)
                                          : ln.run_grad<float>(dl, layout, dkappa, lambda_out);
  ctx->launches = ln.count;
  if (rc) return rc;
  if (o->profile) {
    CK(cudaStreamSynchronize(s));
    ctx->prof.assign(F_COUNT, ProfRecHost());
    for (const ProfRec& r : recs) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      ctx->prof[r.fam].launches++;
      ctx->prof[r.fam].ms += ms;
      ctx->prof[r.fam].bytes += r.bytes;
    }
    ctx->prof_valid = true;
  }
  return MLEV_OK;
}

const double* kappa_device_src(mlev_ctx* ctx, void* ws) {
  const Plan& P = ctx->plan;
  if (P.kappa_kind == MLEV_KAPPA_ONE) return nullptr;
  if (P.kappa_on_device) return P.kappa_dev;
  return at<double>(ws, P.w_kstage);
}

}  // namespace

extern "C" {

void mlev_opts_default(mlev_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MLEV_PREC_MIXED;
  o->vcycles = 4;
  o->refine_passes = 2;
  o->strip_vcycles = 4;
  o->pre_smooth = 2;
  o->post_smooth = 2;
  o->coarse_sweeps = 40;
  o->level1_max_iter = 60;
  o->level1_tol = 1e-10;
  o->rr_max_iter = 100;
  o->use_graph = 0;
  o->omega = 1.0;
  o->check_residuals = 0;
  o->fused = 1;
}

int mlev_create(mlev_ctx** out, int device) {
  if (!out) return MLEV_EINVAL;
  *out = nullptr;
  if (device == -1) {  // planning-only context: set-up, validation and sizes, no solves
    mlev_ctx* c = new (std::nothrow) mlev_ctx();
    if (!c) return MLEV_ENOMEM;
    c->device = -1;
    c->uid = g_next_ctx_uid.fetch_add(1);
    *out = c;
    return MLEV_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MLEV_ECUDA;
  mlev_ctx* c = new (std::nothrow) mlev_ctx();
  if (!c) return MLEV_ENOMEM;
  c->device = device;
  c->uid = g_next_ctx_uid.fetch_add(1);
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) {
    delete c;
    return MLEV_ECUDA;
  }
  *out = c;
  return MLEV_OK;
}

void mlev_destroy(mlev_ctx* ctx) {
  if (!ctx) return;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

const char* mlev_last_error(const mlev_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mlev_set_domain(mlev_ctx* ctx, int ncx, int ncy, double x0, double y0, double H, const uint8_t* cell_in) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  if (ncx < 2 || ncy < 2 || ncx > 64 || ncy > 64 || !(H > 0) || !cell_in)
    return fail(ctx, MLEV_EINVAL, "domain: need 2 <= ncx, ncy <= 64, H > 0 and a cell mask");
  Plan& P = ctx->plan;
  P.ncx = ncx;
  P.ncy = ncy;
  P.x0 = x0;
  P.y0 = y0;
  P.H = H;
  P.cell_in.assign(cell_in, cell_in + (size_t)ncx * ncy);
  for (auto& v : P.cell_in) v = v ? 1 : 0;
  bool any = false;
  for (auto v : P.cell_in) any = any || v;
  if (!any) return fail(ctx, MLEV_EINVAL, "domain has no cell");
  P.has_domain = true;
  P.has_partition = false;
  ctx->version++;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_set_partition(mlev_ctx* ctx, int m, const int32_t* owner, const int32_t* overlap, double delta,
                       int glue_mode) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  Plan& P = ctx->plan;
  if (!P.has_domain) return fail(ctx, MLEV_ESTATE, "set the domain first");
  if (m < 1 || !owner || !overlap) return fail(ctx, MLEV_EINVAL, "partition: need m >= 1, cell_owner and overlap");
  if (glue_mode != MLEV_GLUE_PAPER) return fail(ctx, MLEV_EUNSUPPORTED, "only MLEV_GLUE_PAPER is implemented");
  P.m = m;
  P.owner.assign(owner, owner + (size_t)P.ncx * P.ncy);
  P.overlap.assign(overlap, overlap + m);
  P.delta = delta;
  P.glue_mode = glue_mode;
  std::string e = check_partition(P);
  int rc = map_plan_error(ctx, e);
  if (rc) return rc;
  P.has_partition = true;
  ctx->version++;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_set_levels(mlev_ctx* ctx, int n) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  if (n < 2 || n > MLEV_MAX_LEVELS) return fail(ctx, MLEV_EINVAL, "levels: need 2 <= n <= MLEV_MAX_LEVELS");
  Plan& P = ctx->plan;
  if (P.has_forms && P.kappa_kind == MLEV_KAPPA_PER_FINE_ELEM && P.n != n) P.has_forms = false;
  P.n = n;
  P.has_levels = true;
  ctx->version++;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_set_eigenpairs(mlev_ctx* ctx, int q) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  if (q < 1 || q > MLEV_MAX_EIGENPAIRS) return fail(ctx, MLEV_EINVAL, "eigenpairs: need 1 <= q <= MLEV_MAX_EIGENPAIRS");
  Plan& P = ctx->plan;
  P.q = q;
  P.B = P.Breal * q;
  ctx->version++;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_set_forms(mlev_ctx* ctx, int batch, int kappa_kind, const double* kappa, int kappa_on_device) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  Plan& P = ctx->plan;
  if (batch < 1) return fail(ctx, MLEV_EINVAL, "batch must be >= 1");
  if (kappa_kind < MLEV_KAPPA_ONE || kappa_kind > MLEV_KAPPA_PER_FINE_ELEM)
    return fail(ctx, MLEV_EINVAL, "unknown kappa kind");
  if (kappa_kind != MLEV_KAPPA_ONE && !kappa) return fail(ctx, MLEV_EINVAL, "kappa values required");
  if (!P.has_domain) return fail(ctx, MLEV_ESTATE, "set the domain first");
  if (kappa_kind == MLEV_KAPPA_PER_FINE_ELEM && !P.has_levels)
    return fail(ctx, MLEV_ESTATE, "set the levels before per-element kappa");
  P.Breal = batch;
  P.B = batch * P.q;
  P.kappa_kind = kappa_kind;
  P.kappa_on_device = kappa_on_device != 0;
  P.kappa_dev = P.kappa_on_device ? kappa : nullptr;
  P.kappa_host.clear();
  if (kappa_kind != MLEV_KAPPA_ONE && !P.kappa_on_device) {
    size_t cnt = kappa_kind == MLEV_KAPPA_PER_COARSE_CELL
                     ? (size_t)batch * P.ncx * P.ncy
                     : (size_t)batch * ((size_t)P.ncx << P.n) * ((size_t)P.ncy << P.n) * 2;
    P.kappa_host.assign(kappa, kappa + cnt);
    for (size_t i = 0; i < cnt; ++i)
      if (!(P.kappa_host[i] >= 0) || !std::isfinite(P.kappa_host[i]))
        return fail(ctx, MLEV_EINVAL, "kappa must be finite and non-negative");
  }
  P.has_forms = true;
  ctx->version++;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_workspace_size(mlev_ctx* ctx, const mlev_opts* opts, size_t* bytes) {
  MLEV_TRY
  if (!ctx || !bytes) return MLEV_EINVAL;
  if (!opts_valid(opts)) return fail(ctx, MLEV_EINVAL, "invalid options");
  int rc = ensure_plan(ctx, opts);
  if (rc) return rc;
  *bytes = ctx->plan.ws_bytes;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_problem_info(mlev_ctx* ctx, long long* n_fine, long long* n_local_fine, long long* n_strip_fine,
                      int* n_coarse) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  mlev_opts o;
  mlev_opts_default(&o);
  if (ctx->built_precision >= 0) o.precision = ctx->built_precision;
  int rc = ensure_plan(ctx, &o);
  if (rc) return rc;
  const Plan& P = ctx->plan;
  if (n_fine) *n_fine = P.n_fine;
  if (n_local_fine) *n_local_fine = P.lp[P.n].n_local;
  if (n_strip_fine) *n_strip_fine = P.lp[P.n].n_strip;
  if (n_coarse) *n_coarse = P.n_coarse;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_solve(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
               double* lambda_out, double* u_out, mlev_report* rep) {
  MLEV_TRY
  int rc = prepare(ctx, opts, workspace, ws_bytes);
  if (rc) return rc;
  if (!lambda_out) return fail(ctx, MLEV_EINVAL, "lambda_out is required");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, MLEV_ECUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  rc = upload_tables(ctx, workspace, s, false);
  if (rc) return rc;
  rc = solve_impl(ctx, opts, workspace, ws_bytes, s, kappa_device_src(ctx, workspace), lambda_out, u_out);
  if (rc) return rc;
  if (rep) return fill_report(ctx, workspace, s, rep);
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_solve_host(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
                    const double* kappa_host, double* lambda_host, double* u_host, mlev_report* rep) {
  MLEV_TRY
  int rc = prepare(ctx, opts, workspace, ws_bytes);
  if (rc) return rc;
  if (!lambda_host) return fail(ctx, MLEV_EINVAL, "lambda_host is required");
  const Plan& P = ctx->plan;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, MLEV_ECUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  rc = upload_tables(ctx, workspace, s, true);
  if (rc) return rc;
  const double* ksrc = kappa_device_src(ctx, workspace);
  if (kappa_host && P.kappa_kind != MLEV_KAPPA_ONE && P.q > 1)
    return fail(ctx, MLEV_EUNSUPPORTED, "new kappa values per call are not supported with several eigenpairs");
  if (kappa_host && P.kappa_kind != MLEV_KAPPA_ONE) {
    CK(cudaMemcpyAsync(at<char>(workspace, P.w_kstage), kappa_host, P.w_kstage.bytes, cudaMemcpyHostToDevice, s));
    ctx->io_h2d += (long long)P.w_kstage.bytes;
    ksrc = at<double>(workspace, P.w_kstage);
  }
  double* dlam = at<double>(workspace, P.w_out_lam);
  double* du = u_host ? at<double>(workspace, P.w_out_u) : nullptr;
  rc = solve_impl(ctx, opts, workspace, ws_bytes, s, ksrc, dlam, du);
  if (rc) return rc;
  CK(cudaMemcpyAsync(lambda_host, dlam, (size_t)P.B * 8, cudaMemcpyDeviceToHost, s));
  ctx->io_d2h += (long long)P.B * 8;
  if (u_host) {
    const size_t ub = (size_t)P.B * (P.lvl_nx(P.n) + 1) * (P.lvl_ny(P.n) + 1) * 8;
    CK(cudaMemcpyAsync(u_host, du, ub, cudaMemcpyDeviceToHost, s));
    ctx->io_d2h += (long long)ub;
  }
  CK(cudaStreamSynchronize(s));
  if (rep) return fill_report(ctx, workspace, s, rep);
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_grad_workspace_size(mlev_ctx* ctx, const mlev_opts* opts, size_t* bytes) {
  MLEV_TRY
  if (!ctx || !bytes) return MLEV_EINVAL;
  if (!opts_valid(opts)) return fail(ctx, MLEV_EINVAL, "invalid options");
  int rc = ensure_plan(ctx, opts);
  if (rc) return rc;
  *bytes = ctx->plan.ws_grad_bytes;
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

int mlev_grad_kappa(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
                    const double* dlambda, int layout, double* dkappa, double* lambda_out, mlev_report* rep) {
  MLEV_TRY
  int rc = prepare(ctx, opts, workspace, ws_bytes);
  if (rc) return rc;
  const Plan& P = ctx->plan;
  if (ws_bytes < P.ws_grad_bytes)
    return fail(ctx, MLEV_ENOMEM, "workspace too small for the adjoint: need " + std::to_string(P.ws_grad_bytes) +
                                      " bytes (mlev_grad_workspace_size)");
  if (P.q > 1) return fail(ctx, MLEV_EUNSUPPORTED, "the gradient is implemented for one eigenpair");
  if (!dlambda || !dkappa) return fail(ctx, MLEV_EINVAL, "dlambda and dkappa are required");
  if (layout != MLEV_GRAD_FINE_ELEM && layout != MLEV_GRAD_COARSE_CELL)
    return fail(ctx, MLEV_EINVAL, "unknown gradient layout");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, MLEV_ECUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  rc = upload_tables(ctx, workspace, s, false);
  if (rc) return rc;
  rc = grad_impl(ctx, opts, workspace, s, kappa_device_src(ctx, workspace), dlambda, layout, dkappa, lambda_out);
  if (rc) return rc;
  if (rep) return fill_report(ctx, workspace, s, rep);
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

}  // extern "C"

extern "C" int mlev_profile_read(mlev_ctx* ctx, mlev_kernel_stat* out, int capacity, int* count) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  if (!ctx->prof_valid) return fail(ctx, MLEV_ESTATE, "no profiled solve has completed");
  if (count) *count = F_COUNT;
  for (int i = 0; i < F_COUNT && i < capacity && out; ++i) {
    std::memset(&out[i], 0, sizeof(out[i]));
    std::snprintf(out[i].name, sizeof(out[i].name), "%s", kFamName[i]);
    out[i].launches = ctx->prof[i].launches;
    out[i].ms = ctx->prof[i].ms;
    out[i].bytes = ctx->prof[i].bytes;
  }
  return MLEV_OK;
  MLEV_CATCH(ctx)
}

// ---------------------------------------------------------------------------------
// Workspace-free entry point. Its scratch is this fixed device array (one per GPU that
// loads the library, alive until exit); host code must not use the symbol as an
// address, so its device address is looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_workspace[MLEV_NOALLOC_WORKSPACE_BYTES];

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[256] = {nullptr};
// whose plan tables the array of each device holds: context uid and plan generation
// (0 = none yet); a context that finds its own tables there skips the copy
unsigned long long g_noalloc_owner[256] = {0};
long long g_noalloc_gen[256] = {0};
}  // namespace

extern "C" int mlev_solve_noalloc(mlev_ctx* ctx, const mlev_opts* opts, void* stream, double* lambda_out,
                                  double* u_out, mlev_report* rep) {
  MLEV_TRY
  if (!ctx) return MLEV_EINVAL;
  if (ctx->device < 0) return fail(ctx, MLEV_ESTATE, "planning-only context (device -1) cannot solve");
  if (ctx->device >= 256) return fail(ctx, MLEV_EUNSUPPORTED, "device index above 255");
  if (!opts_valid(opts)) return fail(ctx, MLEV_EINVAL, "invalid options");
  int rc = ensure_plan(ctx, opts);
  if (rc) return rc;
  if (ctx->plan.ws_bytes > (size_t)MLEV_NOALLOC_WORKSPACE_BYTES)
    return fail(ctx, MLEV_ENOMEM,
                "problem needs " + std::to_string(ctx->plan.ws_bytes) +
                    " bytes of workspace; the no-allocation entry point holds at most " +
                    std::to_string((size_t)MLEV_NOALLOC_WORKSPACE_BYTES) + " bytes (use mlev_solve with a larger one)");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, MLEV_ECUDA, "cudaSetDevice");
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[ctx->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_workspace);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(no-allocation workspace)");
      g_noalloc_ptr[ctx->device] = p;
    }
    ws = g_noalloc_ptr[ctx->device];
  }
  rc = prepare(ctx, opts, ws, MLEV_NOALLOC_WORKSPACE_BYTES);
  if (rc) return rc;
  if (!lambda_out) return fail(ctx, MLEV_EINVAL, "lambda_out is required");
  cudaStream_t s = (cudaStream_t)stream;
  {
    // the array is shared by every context: copy this problem's tables (and staged kappa) in
    // unless the last copy into it was this context's, for its current plan
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const bool mine = g_noalloc_owner[ctx->device] == ctx->uid && g_noalloc_gen[ctx->device] == ctx->plan_gen;
    if (!mine) {
      g_noalloc_owner[ctx->device] = 0;  // stays unowned if the copy fails
      rc = upload_tables(ctx, ws, s, true);
      if (rc) return rc;
      g_noalloc_owner[ctx->device] = ctx->uid;
      g_noalloc_gen[ctx->device] = ctx->plan_gen;
    }
  }
  rc = solve_impl(ctx, opts, ws, MLEV_NOALLOC_WORKSPACE_BYTES, s, kappa_device_src(ctx, ws), lambda_out, u_out);
  if (rc) return rc;
  if (rep) return fill_report(ctx, ws, s, rep);
  return MLEV_OK;
  MLEV_CATCH(ctx)
}
