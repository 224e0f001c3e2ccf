// Internal data structures shared by the host planner (plan.cpp), the kernels and
// the C-ABI layer. Plain old data only, so the same structs live in host and device
// memory.
#pragma once

#include <stddef.h>
#include <stdint.h>

#define MLEV_MAX_TOTAL_LEVELS 16  // level-1 job may coarsen below T_H; absolute levels in [-6, 10]
#define MLEV_LMIN (-6)

// One grid of one multigrid job at one level. A job is a rectangular window of the
// level-l lattice (a subdomain Omega_j, the strip G_{m+1}, or the whole domain for the
// level-1 eigenproblem) together with a region mask that says which interior nodes
// are unknowns.
struct GridDesc {
  int nx, ny;        // cells; nodes 0..nx x 0..ny, the outer ring is never an unknown
  int pitch;         // row pitch in elements
  int ox, oy;        // lattice coordinates of node (0,0) in the global level-`level` lattice
  int level;         // absolute level (mesh size H / 2^level), may be negative
  int problem;       // batch member
  int full;          // 1: every strictly interior node is an unknown (no region lookups)
  int rshift;        // level - (level of the region grid)
  int rnx, rny;      // region grid size in region cells
  int job;           // owning job
  int depth;         // 0 = finest grid of the job
  long long roff;    // byte offset of the region grid in the region pool
  long long off;     // element offset of node (0,0) in the X / F pools
  long long off64;   // element offset in the FP64 pools (finest grid only, else -1)
  int tmap;          // first of this grid's 3 TMA tensor maps (x fine box, f fine box, x coarse box), -1 if none
  int pad_;
};

// TMA boxes of the fused multigrid kernels (nodes): the fine box covers a 64 x 64 output
// tile with a halo of up to 8 columns and 6 rows; the coarse box covers the coarse nodes
// the prolongation of such a tile (halo <= 4) reads.
#define MLEV_TMA_FBW 80
#define MLEV_TMA_FBH 76
#define MLEV_TMA_FOX 8   // fine box starts at (x0 - 8, y0 - 6)
#define MLEV_TMA_FOY 6
#define MLEV_TMA_CBW 40
#define MLEV_TMA_CBH 38
#define MLEV_TMA_COX 4   // coarse box starts at (x0/2 - 4, y0/2 - 3)
#define MLEV_TMA_COY 3
#define MLEV_TMAP_BYTES 128

// Output tile of the register-blocked fused multigrid kernels (kern_mgreg.cu): 112 x 52
// nodes, origins multiples of the tile size (even, and x a multiple of 4 for float4 rows).
#define MLEV_SUBEIG_SMEM_MAX (220 * 1024)  // shared memory limit of the subspace eigensolver
#define MLEV_RTILE_W 112
#define MLEV_RTILE_H 52

struct Tile {  // a block of nodes of one grid: origin (x0, y0), size fixed by the kernel
  int grid;
  int x0, y0;
};

// Device view of the coefficient kappa.
struct KappaDev {
  int kind;                          // MLEV_KAPPA_*
  int ncx, ncy;                      // T_H
  const double* coarse;              // kind PER_COARSE_CELL: [B][ncy][ncx]
  const double* lvl;                 // per-level triangle values (kinds 1 with level<0, and 2)
  const float* coarse_f;             // FP32 copies of coarse and lvl, read by the FP32 multigrid
  const float* lvl_f;
  long long lvl_off[MLEV_MAX_TOTAL_LEVELS];     // element offset of level (l - MLEV_LMIN)
  long long lvl_bstride[MLEV_MAX_TOTAL_LEVELS]; // elements per batch member at that level
};

// Everything a kernel needs to interpret grids.
struct DevGeom {
  const GridDesc* grids;
  const uint8_t* regions;   // region pool
  const int16_t* qlabel;    // [4*ncy][4*ncx]: -1 outside Omega, 0 strip, j+1 inside G_j
  const uint8_t* cell_in;   // [ncy][ncx]
  const int* sub_top;       // [B*m] grid index of the finest grid of subdomain j of problem b (current level)
  const unsigned char* tmaps;  // TMA tensor maps, MLEV_TMAP_BYTES each (64-byte aligned)
  unsigned long long* status;  // device status bits (MLEV_ST_*), problem 0's flags slot
  int ncx, ncy, m;
  double H;
  KappaDev kap;
};

// Global per-level field layout (per batch member): rows 0..NY_l, pitch gpitch[l].
struct GlobalLayout {
  int nx[MLEV_MAX_TOTAL_LEVELS];      // cells at level l (index l - MLEV_LMIN)
  int ny[MLEV_MAX_TOTAL_LEVELS];
  int pitch[MLEV_MAX_TOTAL_LEVELS];
  long long bstride;                  // elements per batch member (sized for the finest level)
};

// Device status bits.
#define MLEV_ST_LEVEL1_NOCONV 1
#define MLEV_ST_RR_NOCONV 2
#define MLEV_ST_RR_BREAKDOWN 4
#define MLEV_ST_NONFINITE 8
#define MLEV_ST_TIMEOUT 16  // a bounded wait on a TMA transaction barrier gave up
#define MLEV_ST_ADJ_NOCONV 32  // the level-1 adjoint solve reached its iteration cap

// Per-problem status record (long long slots), stride mlev_stat_stride(n).
#define MLEV_STAT_L1_IT 0     // level-1 iterations
#define MLEV_STAT_L1_RES 1    // level-1 final relative residual (double bits)
#define MLEV_STAT_FLAGS 2     // MLEV_ST_* bits
#define MLEV_STAT_RR_IT 4     // + L: Rayleigh-Ritz iterations on level L
#define MLEV_STAT_LOC_RES(n) (4 + ((n) + 1))        // + L: max relative residual of the local solves
#define MLEV_STAT_STRIP_RES(n) (4 + 2 * ((n) + 1))  // + L: relative residual of the G_{m+1} solve
static inline int mlev_stat_stride(int n) { return 4 + 3 * (n + 1); }

/* Bytes per batch member of the Rayleigh-Ritz factors prepared ahead of a level (mixed
   precision, row-blocked factors): the shift sigma (double), a flag (int, 1 = valid), padding
   to 16 bytes, then P_I^{-1}, W_I and W_I^T as BS x (BS + 4) float tiles for the
   nhb / (bw - 1) grid rows (BS = 16 or 32). 0 when the coarse system has no row-blocked
   form. */
static inline size_t mlev_rr_prefactor_stride(int nhb, int bw) {
  const int bsz = bw - 1;
  if (bsz <= 0 || bsz > 32 || nhb <= 0) return 0;
  const size_t bs = bsz <= 16 ? 16 : 32, ts = bs * (bs + 4);
  return 16 + ((3 * (size_t)(nhb / bsz) * ts * 4 + 15) / 16) * 16;
}
