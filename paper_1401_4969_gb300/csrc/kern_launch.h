// Host-callable launchers of the device kernels (one per kernel family). Every
// launcher enqueues on the given stream and never synchronizes.
#pragma once

#include "kern_common.cuh"

namespace mlev {

// ---- multigrid (kern_mg.cu), T = float (mixed) or double (plain FP64) ----
template <typename T>
void launch_smooth(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int color, double omega,
                   cudaStream_t s);
template <typename T>
// black_zero: the fine grid's last half-sweep was black with omega = 1 (k_restrict)
void launch_restrict(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, int black_zero, cudaStream_t s);
template <typename T>
// red_only: the next half-sweep is black with omega = 1 (k_prolong)
void launch_prolong(const DevGeom& G, const Tile* tiles, int n, T* X, int red_only, cudaStream_t s);
template <typename T>
void launch_coarsest(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int sweeps, double omega,
                     cudaStream_t s);
template <typename T>
void launch_coarse_inverse(const DevGeom& G, const Tile* tiles, int n, T* inv, int nd_max, cudaStream_t s);
template <typename T>
void launch_coarsest_direct(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, const T* inv, int nd_max,
                            cudaStream_t s);
size_t coarsest_smem_bytes(int kappa_kind, int nodes, int tsize);  // staged coarsest kernel; limit 220 KiB
template <typename T>
void launch_coarsest_smem(const DevGeom& G, const Tile* tiles, int n, int max_nodes, T* X, const T* F, int sweeps,
                          double omega, cudaStream_t s);
void launch_job_resnorm(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, const double* E, int use64,
                        const double* R, double* acc, cudaStream_t s);
void launch_resnorm_finalize(const double* acc, int B, int m, int subdomains, long long* stat, int stat_stride,
                             int slot, cudaStream_t s);
template <typename T>
void launch_gather(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* X, T* F, double* X64,
                   const double* R, cudaStream_t s);
template <typename T>
void launch_accumulate(const DevGeom& G, const Tile* tiles, int n, T* X, double* X64, cudaStream_t s);
template <typename T>
void launch_refine_residual(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* F,
                            const double* X64, const double* R, cudaStream_t s);

// ---- fused multigrid (kern_mgfused.cu); nu in {1, 2} ----
constexpr int kTailSmemMax = 200 * 1024;
template <typename T>
void launch_mg_down(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, int nu, double omega, cudaStream_t s);
template <typename T>
void launch_mg_up(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int nu, double omega, cudaStream_t s);
template <typename T>
void launch_mg_tail(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, const T* inv, int nd_max, int nlev,
                    int pre, int post, int csweeps, double omega, int load_x, size_t smem, cudaStream_t s);

// ---- register-blocked fused multigrid, FP32 (kern_mgreg.cu); tiles of MLEV_RTILE_W x
// MLEV_RTILE_H nodes; full = every grid of the tile list has no region mask ----
bool rkernels_support(int kappa_kind, int level, int pre, int post, double omega);  // per depth (grid level)
// down: nu sweeps on depth d (x read from X, smoothed x written to XS), residual, restriction to
// depth d + 1 (f and x = 0 there, in F and X)
void launch_rdown(const DevGeom& G, const Tile* tiles, int n, int full, float* X, float* XS, float* F, int nu,
                  int black_zero, cudaStream_t s);
// up: x = XS + P x_c (x_c from X at depth d + 1), nu sweeps, written to X
void launch_rup(const DevGeom& G, const Tile* tiles, int n, int full, const float* XS, float* X, const float* F, int nu,
                int red_only, cudaStream_t s);
// ---- several eigenpairs (kern_multi.cu): q virtual batch members per problem ----
constexpr int kSubEigSmemMax = MLEV_SUBEIG_SMEM_MAX;
struct SubEigArgs {
  int q, s;                 // eigenpairs wanted, block size (q <= s <= 16)
  int nb, bwk, bwm;         // band rows; half bandwidth of K (factored, <= 31) and of the band storage
  int nbord;                // border size: 0 (level 1) or q (Rayleigh-Ritz on V_{0H} + span{u~_i})
  const double* K;          // [Breal] bands [nb][bwm + 1] (entry [r][d] = A(r, r - d)), stride kstride
  const double* M;
  long long kstride, mstride;
  const double* Ga;         // [Breal][nbord][nb] border columns of A and B
  const double* Gb;
  const double* Aq;         // [Breal][nbord][nbord]
  const double* Bq;
  double* X;                // [Breal][s][nb + nbord]: out, B-orthonormal Ritz vectors (ascending)
  double* Y;
  double* AY;
  double* BY;
  double* Z;                // [Breal][nbord][nb]
  double* theta;            // [Breal][s]: out, Ritz values
  int max_iter;
  double tol;               // FP64 Rayleigh-Ritz from the step the q wanted Ritz values change by <= tol
  double rtol;              // stop when every wanted Ritz pair has ||A x - theta B x|| <= rtol ||theta B x||
  int init_border;          // 1: start from the border unit vectors
  long long* stat;          // per virtual member b q + i
  int stat_stride, it_slot;
  int res_slot;             // stat slot for the final relative residual (as double bits), or -1
  int noconv_flag;
};
void launch_band_level(const DevGeom& G, int Breal, int q, int l, double* K, double* M, cudaStream_t s);
void launch_cross_gram(const DevGeom& G, const GlobalLayout& gl, int L, int Breal, int q, const double* ut, double* out,
                       cudaStream_t s);
void launch_border_prep(const DevGeom& G, int Breal, int q, const double* partials, const double* cross, double* Ga,
                        double* Gb, double* Aq, double* Bq, cudaStream_t s);
void launch_sub_eig(const DevGeom& G, const SubEigArgs& a, int Breal, cudaStream_t s);
void launch_level1_multi_out(const DevGeom& G, const GlobalLayout& gl, int Breal, int q, int s_, const double* X,
                             const double* theta, double* ut1, double* lam, int lam_stride, double* c, double* c0,
                             cudaStream_t s);
void launch_rr_multi_out(const DevGeom& G, int Breal, int q, int s_, int nb, int bw, int L, int lam_stride,
                         const double* X, const double* theta, const double* MH, long long mstride, const double* Gb,
                         double* c, double* c0, double* D, double* lam, cudaStream_t s);
void launch_combine(const GlobalLayout& gl, int L, int Breal, int q, const double* D, const double* src, double* dst,
                    cudaStream_t s);
// ---- global fields (kern_field.cu) ----
struct LevelArgs {
  int L;                 // current level
  int B;
  const double* ut_prev; // u~ on level L-1 (pitched, level L-1 layout)
  double* ut;            // u~ on level L
  double* uin;           // u_{h_k} embedded in V_{h_L}
  double* r;             // residual / right-hand side field
  const double* c;       // [B][(ncy+1)(ncx+1)] coarse coefficients of u_{h_k}
  const double* c0;      // [B] coefficient of u~ in u_{h_k}
  const double* lam;     // [B][n+1] eigenvalue per level
  int lam_stride;        // n + 1
  double m12;            // h_L^2 / 12, the weight of the consistent mass stencil on level L
};
void launch_interp(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, cudaStream_t s);
void launch_rhs(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, cudaStream_t s);
// glue: E = FP64 local solutions (pool base); use64 selects GridDesc::off64 (mixed) or ::off (FP64 mode);
// E32 (nullable) = the FP32 pool, read instead of E when it holds the whole solution
void launch_glue(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const double* E, int use64,
                 const float* E32, cudaStream_t s);
template <typename T>
void launch_strip_rhs(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const Tile* tiles, int n, T* X,
                      T* F, double* X64, cudaStream_t s);
void launch_strip_update(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const Tile* tiles, int n,
                         const double* E, int use64, const float* E32, cudaStream_t s);
// Rayleigh-Ritz factors prepared by one extra block per batch member of the inner-product
// kernel (rr_prefactor_block); K_H, M_H [B][nhb][bw+1], out [B][stride].
struct RRPrefactor {
  const double* KH;
  const double* MH;
  int nhb, bw;
  unsigned char* out;
  long long stride;
};
void launch_aug(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, double* partials,
                const RRPrefactor* pf, cudaStream_t s);  // pf nullable
void launch_output_u(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* c,
                     const double* c0, double* u_out, cudaStream_t s);
void launch_kappa_copy_fine(const KappaDev& kv, int n, int B, const double* src, double* lvl, float* lvl_f,
                            cudaStream_t s);
void launch_kappa_to_f(long long count, const double* src, float* dst, cudaStream_t s);
void launch_kappa_average(const KappaDev& kv, int l, int B, double* lvl, float* lvl_f, cudaStream_t s);
void launch_band_setup(const DevGeom& G, int B, int nhb, int bw, double* KH, double* MH, cudaStream_t s);
void launch_lambda_out(int B, int n, const double* lam, double* out, cudaStream_t s);

// ---- eigen solvers (kern_eig.cu) ----
struct Level1Args {
  int B;
  int grid_begin, nlev;  // level-1 job grids of problem b: grid_begin + b * nlev + depth
  double* vec;           // 10 FP64 vectors per problem, each vstride elements
  long long vstride;     // elements per vector (per problem); problem b at vec + b * 10 * vstride
  void* xpool;           // multigrid pools (T)
  void* fpool;
  int pre, post, coarse_sweeps;
  double omega;
  int max_iter;
  double tol;
  double* ut1;           // output u~_1 = u_{h_1} on level 1, global layout
  double* lam;           // [B][n+1]: writes index 1
  int lam_stride;
  double* c;             // zeroed coarse coefficients
  double* c0;            // set to 1
  long long* stat;       // [B][...] iterations, residual bits
  int stat_stride;
};
template <typename T>
void launch_level1(const DevGeom& G, const GlobalLayout& gl, const Level1Args& a, cudaStream_t s);
// on-chip variant: every vector and grid of the level-1 hierarchy in shared memory
constexpr int kL1SmemMax = 200 * 1024;
size_t level1_smem_bytes(long long nn0, long long tot, int tsize);
template <typename T>
void launch_level1_sm(const DevGeom& G, const GlobalLayout& gl, const Level1Args& a, size_t smem, cudaStream_t s);

struct RRArgs {
  int B, L, n;
  int nhb, bw;
  const double* KH;
  const double* MH;
  double* chol;          // [B][nhb*(bw+1) + 5*nhb] scratch (used when the system does not fit on chip)
  int smem;              // 1: keep the band system in shared memory
  const double* partials;
  double* lam;           // [B][n+1]
  double* c;             // [B][(ncy+1)(ncx+1)]
  double* c0;            // [B]
  long long* stat;
  int stat_stride;
  int max_iter;
  int mixed;             // 1: FP32 band factors with FP64 refinement (k_rr_mixed)
  const double* c_prev;  // coefficients of u_{h_k} (the previous level's eigenvector): warm start
  const double* c0_prev;
  int blocked;           // 1: row-blocked FP32 solves (needs smem), else the warp solve
  unsigned char* pre;    // [B][pre_stride] factors of S(sigma) prepared ahead (mlev_rr_prefactor_stride)
  long long pre_stride;
  int use_pre;           // k_rr_mixed starts from the prepared factors when their flag is set
};
void launch_rr(const DevGeom& G, const RRArgs& a, cudaStream_t s);
size_t rr_prefactor_smem(int nhb, int bw);  // shared memory of rr_prefactor_block
size_t rr_smem_bytes(int nhb, int bw);
size_t rr_mixed_smem_bytes(int nhb, int bw, int blocked);
int rr_mixed_supported(int nhb, int bw);
constexpr int kRRSmemMax = 200 * 1024;

// ---- adjoint of Algorithm 4.2 (kern_adj.cu) ----
// A field of level L written as sum_i c_i phi_i^H + s * f (the basis {coarse hats, u~} of
// the Rayleigh-Ritz step): c nullable ([B][ncoef], stride cstride), s nullable (read as 1),
// f a global level-L field.
struct AugField {
  const double* c;
  long long cstride;
  const double* s;
  int sstride;
  const double* f;
};
struct GradLevels {                 // per-level triangle gradients [B][ny_l][nx_l][2]
  long long off[MLEV_MAX_LEVELS + 1];  // element offset of level l (1..n)
};
// Per-problem coefficients the Rayleigh-Ritz adjoint hands to the field kernels:
// [zc | kac | mac] coarse vectors (ncoef each) then kAdjScal scalars.
constexpr int kAdjScal = 8;
enum { ADJ_CU = 0, ADJ_ZU, ADJ_KAU, ADJ_MAU, ADJ_LAMBAR, ADJ_LAM, ADJ_SC, ADJ_SIGMA };
struct RRAdjArgs {
  int B, L, n;
  int nhb, bw;
  const double* KH;
  const double* MH;
  double* scratch;       // [B][nhb*(bw+1) + 10*nhb] (used when the system does not fit on chip)
  int smem;
  const double* partials;  // k_aug partials of u~_L
  const double* part2;     // k_cbar partials of ubar
  const double* lam;       // [B][n+1]
  const double* lambar;    // [B][n+1]
  const double* c;         // coefficients of u_L
  const double* c0;
  double* coef;            // [B][cstride]
  int cstride;
  long long* stat;
  int stat_stride;
};
size_t rr_adj_smem_bytes(int nhb, int bw);
struct Level1AdjArgs {
  int B;
  int grid_begin, nlev;
  double* vec;
  long long vstride;
  void* xpool;
  void* fpool;
  int pre, post, coarse_sweeps;
  double omega;
  int max_iter;
  double tol;
  const double* ut1;     // u_{h_1}, global level-1 layout
  const double* ubar1;   // its adjoint
  const double* lam;     // [B][n+1]
  int lam_stride;
  double* zout;          // solution z, global level-1 layout
  long long* stat;
  int stat_stride;
};
template <typename T>
void launch_gather_masked(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* X, T* F, double* X64,
                          const double* R, cudaStream_t s);
template <typename T>
void launch_refine_residual_masked(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* F,
                                   const double* X64, const double* R, cudaStream_t s);
void launch_cbar(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* ubar,
                 double* part2, cudaStream_t s);
void launch_rr_adj(const DevGeom& G, const RRAdjArgs& a, cudaStream_t s);
void launch_adj_ut(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* ubar,
                   const double* coef, int cstride, double* utbar, cudaStream_t s);
void launch_grad_aug(const DevGeom& G, const GlobalLayout& gl, int L, int B, const AugField& f1, const AugField& f2,
                     const double* w11, int w11_stride, double w12, double* gl_lvl, cudaStream_t s);
void launch_grad_pair(const DevGeom& G, const GlobalLayout& gl, int L, int B, double w, const double* a,
                      const double* b, double* gl_lvl, cudaStream_t s);
void launch_strip_adj_post(const DevGeom& G, const GlobalLayout& gl, int L, int B, double* utbar, const double* sbar,
                           cudaStream_t s);
void launch_grad_local(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* T_, const double* E,
                       int use64, const double* uin, double* gl_lvl, cudaStream_t s);
void launch_rbar(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* T_, int use64, double* rbar,
                 cudaStream_t s);
int adj_uin_blocks(const GlobalLayout& gl, int L);
void launch_adj_uin(const DevGeom& G, const GlobalLayout& gl, int L, int B, double* utbar, const double* sbar,
                    const double* rbar, const double* uin, const double* lam, int lam_stride, double* lbpart,
                    int nblk_stride, cudaStream_t s);
void launch_lambar_finalize(int B, int nblk, int nblk_stride, const double* lbpart, double* lambar, int lam_stride,
                            int k, cudaStream_t s);
void launch_lambar_init(int B, int n, const double* dl, double* lambar, cudaStream_t s);
void launch_restrict_adj(const DevGeom& G, const GlobalLayout& gl, int k, int B, const double* fine, double* coarse,
                         cudaStream_t s);
template <typename T>
void launch_level1_adj(const DevGeom& G, const GlobalLayout& gl, const Level1AdjArgs& a, cudaStream_t s);
void launch_grad_spread(const DevGeom& G, const GlobalLayout& gl, int n, int B, const GradLevels& lv,
                        const double* glbase, int layout, double* out, cudaStream_t s);

}  // namespace mlev
