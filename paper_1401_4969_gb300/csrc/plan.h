// Host planner: validates the problem setup, derives the decomposition sets of
// Section 4 (D_j, Omega_j, closed G_j, G_{m+1}) and lays out every device table and
// buffer inside the caller's workspace.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "../../include/mlev.h"
#include "mlev_internal.h"

namespace mlev {

struct TileList {
  long long off = 0;   // first tile in the tile table
  int count = 0;
  long long unk = 0;   // unknown nodes of the grids covered (for the traffic model)
};

// Byte range of one workspace region.
struct Span {
  size_t off = 0;
  size_t bytes = 0;
};

struct LevelPlan {                      // correction level L = k + 1
  int grid_begin = 0, grid_end = 0;     // grids of this level in Plan::grids
  std::vector<TileList> sub;            // node tiles of the depth-d grids of all subdomain jobs, d = 0..L
  std::vector<TileList> strip;          // node tiles of the depth-d strip grids, d = 0..L-2
  TileList sub_coarsest;                // one tile per subdomain job: (coarsest grid, 0, 0)
  TileList strip_coarsest;
  TileList sub_top;                     // one tile per subdomain job: (finest grid, 0, 0)
  int sub_top_off = 0;                  // offset of this level's [B*m] table in Plan::sub_top
  long long pool_elems = 0;             // X/F pool elements used
  long long pool64_elems = 0;           // X64 pool elements used
  long long n_local = 0, n_strip = 0;   // unknowns per problem
  long long n_free = 0;                 // free nodes of the level-L lattice per problem
  // fused multigrid: 64x64 tiles (only tiles with unknowns) for depths above the tail,
  // and the tail (one block per job from depth *_dt down to the coarsest grid)
  std::vector<TileList> sub_f, strip_f;
  int sub_dt = 0, strip_dt = 0;          // first tail depth (= number of depths + 1 if no tail fits)
  TileList sub_tail, strip_tail;
  size_t sub_tail_smem = 0, strip_tail_smem = 0;
  // register-blocked fused kernels: MLEV_RTILE_W x MLEV_RTILE_H tiles (only tiles with
  // unknowns) of the depths above the tail, and whether every grid of a depth is full
  std::vector<TileList> sub_r, strip_r;
  std::vector<int> sub_r_full, strip_r_full;
};

constexpr int kDirectMax = 128;         // largest coarsest window solved with a dense inverse
constexpr int kFusedTile = 64;          // output tile edge of the fused down / up kernels
constexpr size_t kTailBudget = 160 * 1024;  // shared memory allowed to one tail block

struct Plan {
  // ---- inputs ----
  int ncx = 0, ncy = 0;
  double x0 = 0, y0 = 0, H = 0;
  std::vector<uint8_t> cell_in;
  int m = 0;
  std::vector<int32_t> owner, overlap;
  double delta = 0;
  int glue_mode = 0;
  int n = 0;
  int B = 0;                               // batch members the kernels see: Breal * q
  int Breal = 0;                           // problems of the caller's batch
  int q = 1;                               // smallest eigenpairs per problem (virtual members b q + i)
  int kappa_kind = 0;
  std::vector<double> kappa_host;
  const double* kappa_dev = nullptr;
  bool kappa_on_device = false;
  bool has_domain = false, has_partition = false, has_levels = false, has_forms = false;

  // ---- derived ----
  std::vector<std::array<int, 4>> D, Om;   // cell rectangles [x0, x1) x [y0, y1)
  std::vector<std::array<int, 4>> G;       // closed G_j in quarter-lattice nodes [x0, x1] x [y0, y1]
  std::vector<int16_t> qlabel;             // [4ncy][4ncx]
  int l1_lc = 0;                           // coarsest level of the level-1 hierarchy (<= 0)
  GlobalLayout glay{};
  std::vector<GridDesc> grids;
  std::vector<Tile> tiles;
  std::vector<uint8_t> regions;
  std::vector<int> sub_top;
  std::vector<LevelPlan> lp;               // indexed by L, valid for 2..n
  int l1_grid_begin = 0, l1_nlev = 0;      // level-1 job grids of problem b start at l1_grid_begin + b*l1_nlev
  std::vector<TileList> l1_tiles;          // unused (level 1 runs in one block per problem)
  long long l1_pool_elems = 0;
  long long n_fine = 0;
  int n_coarse = 0;
  int nhb = 0, bw = 0;                     // coarse band system: rows (ncx-1)(ncy-1), half bandwidth
  int sub_direct = 0;                      // subdomain coarsest grids solved by a dense inverse
  int nd_max = 0;                          // largest coarsest-window size (interior nodes) of a subdomain
  int strip_lvl = 2;                       // level of the strip's coarsest grid (1 if G_{m+1} is a union of T_{h_1} cells)
  int strip_coarse_nodes = 0;              // nodes of the strip's coarsest grid
  int n_tmap_grids = 0;                    // grids carrying TMA tensor maps (3 maps each)

  // ---- workspace layout (depends on opts) ----
  int tsize = 4;
  int tail_nodes = 0;                      // cap on the nodes of a tail's first grid (0: shared-memory budget only)
  Span w_grids, w_tiles, w_regions, w_qlabel, w_cellin, w_subtop;
  Span w_kstage, w_klvl, w_klvl_f, w_kcf, w_band, w_ut[2], w_uin, w_r, w_l1vec, w_l1pool[2];
  Span w_x, w_f, w_x64, w_aug, w_lam, w_c, w_c0, w_stat, w_jobnorm, w_chol, w_out_lam, w_out_u, w_cinv, w_tmaps;
  Span w_rrpre;  // Rayleigh-Ritz factors prepared ahead of a level (mixed precision only)
  Span w_xs;     // smoothed x of the register-blocked down kernels (FP32, same layout as w_x)
  // several eigenpairs (q > 1): level-1 band pencil, subspace blocks, bordered pencil, D
  int msub = 0;                            // block size of the subspace iteration
  int m_nb1 = 0;                           // level-1 band rows
  Span w_mk1, w_mm1, w_mX, w_mY, w_mAY, w_mBY, w_mZ, w_mGa, w_mGb, w_mAq, w_mBq, w_mD, w_mth, w_mcross;
  size_t ws_bytes = 0;
  size_t tables_bytes = 0;
  // adjoint (mlev_grad_kappa): extra regions after the solve's, up to ws_grad_bytes
  Span g_ck_ut, g_ck_c, g_ck_c0, g_ubar[2], g_utbar, g_sbar, g_rbar, g_tbuf, g_gl, g_coef, g_part2, g_lbpart,
      g_lambar, g_rrscr;
  long long gl_off[MLEV_MAX_LEVELS + 1] = {0};  // element offset of level l's triangle gradients in g_gl
  int adj_nblk = 0;                              // partial-sum slots per problem (largest level grid)
  size_t ws_grad_bytes = 0;
  KappaDev kap_template{};  // offsets relative to the workspace base

  std::string build(const mlev_opts& o);   // "" on success, else a message
  bool ready() const { return has_domain && has_partition && has_levels && has_forms; }

  int lvl_nx(int l) const { return glay.nx[l - MLEV_LMIN]; }
  int lvl_ny(int l) const { return glay.ny[l - MLEV_LMIN]; }
  int lvl_pitch(int l) const { return glay.pitch[l - MLEV_LMIN]; }
};

// Shared memory of the subspace eigensolver of several eigenpairs (kern_multi.cu) for a band
// of nb rows, factored half bandwidth bwk and block size s.
size_t sub_eig_smem_bytes(int nb, int bwk, int s);

// Validation helpers used by the C ABI (return "" if fine).
std::string check_partition(Plan& p);
long long grid_unknowns(const Plan& p, const GridDesc& g);

}  // namespace mlev
