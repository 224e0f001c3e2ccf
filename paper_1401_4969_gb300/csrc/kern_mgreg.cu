// Register-blocked fused multigrid kernels (FP32) for the masked SPD problems of
// Algorithm 4.1: the auxiliary problems on Omega_j (Eq. Aux_Problem) and the G_{m+1}
// problem (Eq. G_m+1_Problem). Same operations as k_mg_down / k_mg_up (kern_mgfused.cu)
// -- red-black Gauss-Seidel sweeps, residual, restriction P^T r, prolongation x += P x_c
// -- with the grid values held in registers instead of shared memory:
//
// * A block of 8 warps covers a 128 x 64 box of one grid; warp w holds rows 8w .. 8w+7 of
//   the box and lane l holds columns 4l .. 4l+3 of every one of those rows (x and f as float4
//   loads straight from the pools; f stays in registers for kappa = 1 and goes to shared
//   memory for kappa per coarse cell, whose coefficient selection needs the registers for a
//   third block per SM), so a half-sweep reads the north / south
//   neighbours from the thread's own registers, the west / east neighbour across a lane
//   boundary by one warp shuffle per row, and the rows across warp boundaries from a small
//   shared-memory exchange (one barrier per half-sweep).
// * Temporal blocking as in the shared-memory kernels: every half-sweep invalidates one more
//   ring of the box, so the box carries a halo of 8 columns (float4-aligned) and 6 rows
//   around its 112 x 52 output tile (2 NU + 2 <= 6 for NU <= 2).
// * The down kernel reads x from X and writes the smoothed x to the separate pool XS (the
//   up kernel reads XS and writes X): a box never reads values another block of the same
//   launch writes, so results do not depend on the order in which blocks run.
//
// The smoother is plain red-black Gauss-Seidel (omega = 1; the shared-memory kernels serve
// other relaxation factors).
//
// Node (i, j) of the box has colour (i + j) & 1 (0 red, 1 black) in its grid's coordinates;
// the box origin is even in both directions, so the colour of register (q, k) (row q,
// column k) is (q + k) & 1 and every register index below is known at compile time.
#include "kern_launch.h"

namespace mlev {

namespace {

constexpr int kRW = 128;             // box width (nodes)
constexpr int kRR = 8;               // rows per warp
constexpr int kRWarps = 8;           // warps per block
constexpr int kRHX = 8;              // halo columns on each side
constexpr int kRHY = 6;              // halo rows on each side
constexpr int kROW = kRW - 2 * kRHX; // 112 output columns
constexpr int kROH = kRR * kRWarps - 2 * kRHY;  // 52 output rows
static_assert(kROW == MLEV_RTILE_W && kROH == MLEV_RTILE_H, "tile size of the planner");

struct RegTile {
  float v[kRR][4];
};

// Coefficient constant on each coarse cell (these kernels take it on levels l >= 3 only): the
// columns gi0 - 1 .. gi0 + 3 and the rows gj0 - 1 .. gj0 + 7 a thread's stencils touch lie in
// at most two coarse-cell columns X0, X0 + 1 and rows Y0, Y0 + 1 (a cell spans 2^l >= 8
// nodes), so the thread loads those four values once; per node, bits select the cells NE, SE,
// NW, SW of it (the cells of the lower coarse row / column have bit 0).
struct CoarseK {
  float k00, k10, k01, k11;  // k<x><y>: cell (X0 + x, Y0 + y), 0 outside the grid of cells
  unsigned eb, wb;           // bit k: coarse column of gi0 + k (east cells) / of gi0 + k - 1 is X0 + 1
  unsigned nb, sb;           // bit q: coarse row of gj0 + q (north cells) / of gj0 + q - 1 is Y0 + 1
};

template <int KK>
__device__ __forceinline__ CoarseK make_coarse_k(const KappaDev& kv, int p, int l, int gi0, int gj0) {
  CoarseK c{};
  if (KK != MLEV_KAPPA_PER_COARSE_CELL) return c;
  const int X0 = (gi0 - 1) >> l, Y0 = (gj0 - 1) >> l;
  auto kap = [&](int X, int Y) {
    if (X < 0 || Y < 0 || X >= kv.ncx || Y >= kv.ncy) return 0.f;
    return kv.coarse_f[(long long)p * kv.ncx * kv.ncy + Y * kv.ncx + X];
  };
  c.k00 = kap(X0, Y0);
  c.k10 = kap(X0 + 1, Y0);
  c.k01 = kap(X0, Y0 + 1);
  c.k11 = kap(X0 + 1, Y0 + 1);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (((gi0 + k) >> l) != X0) c.eb |= 1u << k;
    if (((gi0 + k - 1) >> l) != X0) c.wb |= 1u << k;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (((gj0 + q) >> l) != Y0) c.nb |= 1u << q;
    if (((gj0 + q - 1) >> l) != Y0) c.sb |= 1u << q;
  }
  return c;
}

// Coefficient weights of the stiffness row of register node (q, k) (global node (gi0 + k,
// gj0 + q) of level l), with the same formulas as edge_weights_t.
template <int KK>
__device__ __forceinline__ EW<float> rweights(const KappaDev& kv, const CoarseK& c, int p, int l, int gi0, int gj0,
                                              int q, int k) {
  static_assert(KK == MLEV_KAPPA_ONE || KK == MLEV_KAPPA_PER_COARSE_CELL, "register kernels: kappa kinds");
  {
    const bool nh = (c.nb >> q) & 1u, sh = (c.sb >> q) & 1u, eh = (c.eb >> k) & 1u, wh = (c.wb >> k) & 1u;
    const float kn0 = nh ? c.k01 : c.k00, kn1 = nh ? c.k11 : c.k10;
    const float ks0 = sh ? c.k01 : c.k00, ks1 = sh ? c.k11 : c.k10;
    const float kne = eh ? kn1 : kn0, knw = wh ? kn1 : kn0, kse = eh ? ks1 : ks0, ksw = wh ? ks1 : ks0;
    EW<float> r;
    r.e = 0.5f * (kne + kse);
    r.n = 0.5f * (kne + knw);
    r.w = 0.5f * (knw + ksw);
    r.s = 0.5f * (kse + ksw);
    return r;
  }
}

// Row exchange between the warps of the block: buf[0][w] = first row of warp w, buf[1][w] =
// its last row. After the barrier warp w reads the row below its first (last row of warp
// w-1) and the row above its last (first row of warp w+1); the outermost warps read zeros
// (the box's outer ring, which no output depends on).
__device__ __forceinline__ void exchange_rows(float4 (*buf)[kRWarps][32], const RegTile& a, float (&below)[4],
                                              float (&above)[4], int w, int lane) {
  buf[0][w][lane] = make_float4(a.v[0][0], a.v[0][1], a.v[0][2], a.v[0][3]);
  buf[1][w][lane] = make_float4(a.v[kRR - 1][0], a.v[kRR - 1][1], a.v[kRR - 1][2], a.v[kRR - 1][3]);
  __syncthreads();
  const float4 b = w > 0 ? buf[1][w - 1][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 t = w < kRWarps - 1 ? buf[0][w + 1][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  below[0] = b.x; below[1] = b.y; below[2] = b.z; below[3] = b.w;
  above[0] = t.x; above[1] = t.y; above[2] = t.z; above[3] = t.w;
}

// One red-black half-sweep of colour C over the thread's registers (C, the row parity and
// the column are compile-time, so each row updates columns k0 and k0 + 2 with one shuffle).
// The coefficient values are passed through an empty asm statement first: the compiler would
// otherwise form the weights of all 32 nodes once and keep them live across the half-sweeps
// (about 128 registers), which spills; recomputing them per node costs a few selects.
__device__ __forceinline__ CoarseK opaque(CoarseK c) {
  asm volatile("" : "+f"(c.k00), "+f"(c.k10), "+f"(c.k01), "+f"(c.k11), "+r"(c.eb), "+r"(c.wb), "+r"(c.nb),
               "+r"(c.sb));
  return c;
}

template <int KK, int C>
__device__ __forceinline__ void rhalf_sweep(RegTile& x, const RegTile& f, const float4* fw, unsigned mask,
                                            const float (&below)[4],
                                            const float (&above)[4], const KappaDev& kv, const CoarseK& ck0, int p,
                                            int l, int gi0, int gj0) {
  const CoarseK ck = KK == MLEV_KAPPA_PER_COARSE_CELL ? opaque(ck0) : ck0;
#pragma unroll
  for (int q = 0; q < kRR; ++q) {
    const int k0 = (C ^ q) & 1;
    float fq[4];
    if constexpr (KK == MLEV_KAPPA_PER_COARSE_CELL) {  // f of row q from shared memory
      const float4 fv = fw[q * 32 + (threadIdx.x & 31)];
      fq[0] = fv.x; fq[1] = fv.y; fq[2] = fv.z; fq[3] = fv.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) fq[k] = f.v[q][k];
    }
    // the row updates columns k0 and k0 + 2: column 0 needs the west neighbour from lane - 1,
    // column 3 the east neighbour from lane + 1 (one shuffle either way)
    float nb;
    if (k0 == 0) nb = __shfl_up_sync(0xffffffffu, x.v[q][3], 1);
    else nb = __shfl_down_sync(0xffffffffu, x.v[q][0], 1);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = k0 + 2 * kk;
      const float xw = k == 0 ? nb : x.v[q][k == 0 ? 0 : k - 1];
      const float xe = k == 3 ? nb : x.v[q][k == 3 ? 3 : k + 1];
      const float xs = q == 0 ? below[k] : x.v[q == 0 ? 0 : q - 1][k];
      const float xn = q == kRR - 1 ? above[k] : x.v[q == kRR - 1 ? kRR - 1 : q + 1][k];
      float nv;  // plain Gauss-Seidel (omega = 1): the node takes the value that zeroes its residual
      if (KK == MLEV_KAPPA_ONE) {
        nv = ((fq[k] + xe) + (xw + xn) + xs) * 0.25f;
      } else {
        const EW<float> w = rweights<KK>(kv, ck, p, l, gi0, gj0, q, k);
        nv = div_diag<float>((fq[k] + w.e * xe) + (w.w * xw + w.n * xn) + w.s * xs, (w.e + w.w) + (w.n + w.s));
      }
      if (mask & (1u << (q * 4 + k))) x.v[q][k] = nv;
    }
  }
}

// Loads rows [r0, r0 + 8) x columns [c0, c0 + 4) of a pitched grid array (zeros outside the
// grid rows / the pitched row).
__device__ __forceinline__ void rload(RegTile& t, const float* base, int pitch, int ny, int c0, int r0) {
  const bool colok = c0 >= 0 && c0 + 3 < pitch;
#pragma unroll
  for (int q = 0; q < kRR; ++q) {
    const int j = r0 + q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (colok && j >= 0 && j <= ny) v = __ldg(reinterpret_cast<const float4*>(base + (long long)j * pitch + c0));
    t.v[q][0] = v.x; t.v[q][1] = v.y; t.v[q][2] = v.z; t.v[q][3] = v.w;
  }
}

// Loads f rows [r0, r0 + 8) x columns [c0, c0 + 4) into the block's shared rows 8 w .. 8 w + 7
// (float4 per lane, zeros outside as rload): f is read once per half-sweep and row, so it
// lives in shared memory and its 32 values leave the thread's registers.
__device__ __forceinline__ void rload_sm(float4* fs, const float* base, int pitch, int ny, int c0, int r0, int w,
                                         int lane) {
  const bool colok = c0 >= 0 && c0 + 3 < pitch;
#pragma unroll
  for (int q = 0; q < kRR; ++q) {
    const int j = r0 + q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (colok && j >= 0 && j <= ny) v = __ldg(reinterpret_cast<const float4*>(base + (long long)j * pitch + c0));
    fs[(w * kRR + q) * 32 + lane] = v;
  }
}

// Unknown mask of the thread's 8 x 4 nodes: bit q * 4 + k. On a grid with a region mask the
// nodes are tested one by one only where some region cell next to the block is outside the
// region (a node is an unknown when its four adjacent cells are in it; with region cells of
// 4 or more nodes the block touches at most 3 x 3 of them, and inside the region interior
// the bounds test alone decides).
template <bool FULL>
__device__ __forceinline__ unsigned rmask(const DevGeom& G, const GridDesc& g, int c0, int r0) {
  bool inside = FULL || g.full;
  if (!inside && g.rshift >= 2) {
    const int ia = max(c0, 1), ib = min(c0 + 3, g.nx - 1), ja = max(r0, 1), jb = min(r0 + kRR - 1, g.ny - 1);
    if (ia > ib || ja > jb) return 0u;
    const int s = g.rshift;
    inside = true;
    for (int cy = (ja - 1) >> s; cy <= (jb >> s); ++cy)
      for (int cx = (ia - 1) >> s; cx <= (ib >> s); ++cx) inside = inside && region_at(G, g, cx, cy);
  }
  unsigned m = 0;
#pragma unroll
  for (int q = 0; q < kRR; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = c0 + k, j = r0 + q;
      const bool u = inside ? (i >= 1 && j >= 1 && i < g.nx && j < g.ny) : is_unknown(G, g, i, j);
      if (u) m |= 1u << (q * 4 + k);
    }
  return m;
}

// Writes the thread's rows that lie in the output tile [x0, x0 + 112) x [y0, y0 + 52) of
// the grid (the columns of lanes 2 .. 29).
__device__ __forceinline__ void rstore(const RegTile& t, float* base, int pitch, int ny, int c0, int r0, int y0,
                                       int lane) {
  if (lane < 2 || lane >= 30 || c0 + 3 >= pitch) return;
#pragma unroll
  for (int q = 0; q < kRR; ++q) {
    const int j = r0 + q;
    if (j < y0 || j >= y0 + kROH || j > ny) continue;
    *reinterpret_cast<float4*>(base + (long long)j * pitch + c0) = make_float4(t.v[q][0], t.v[q][1], t.v[q][2], t.v[q][3]);
  }
}

struct RGrid {  // the fields of a GridDesc the kernels use, read once
  int nx, ny, pitch, ox, oy, level, problem;
  long long off;
};
__device__ __forceinline__ RGrid rgrid(const GridDesc& g) {
  return RGrid{g.nx, g.ny, g.pitch, g.ox, g.oy, g.level, g.problem, g.off};
}

}  // namespace

// Down leg on one tile: NU red-black sweeps (red first), the residual, and its restriction
// to the next coarser grid (f_c = P^T r, x_c = 0) for the coarse nodes of the tile.
template <int KK, int NU, bool FULL>
__global__ void __launch_bounds__(256, KK == MLEV_KAPPA_ONE ? 2 : 3) k_rdown(DevGeom G, const Tile* __restrict__ tiles,
                                                  const float* __restrict__ X, float* XC, float* __restrict__ XS,
                                                  float* F, int black_zero) {
  // kappa = 1: f in registers (2 blocks per SM); kappa per coarse cell: f, then the residual,
  // in shared memory (3 blocks per SM: the coefficient selection needs registers). Each was the
  // faster form on its workload.
  constexpr bool SMF = KK == MLEV_KAPPA_PER_COARSE_CELL;
  __shared__ float4 xbuf[2][2][kRWarps][32];
  extern __shared__ float4 fs[];  // SMF: [64 rows][32 lanes]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Tile t = tiles[blockIdx.x];
  const GridDesc& gd = G.grids[t.grid];
  const RGrid g = rgrid(gd);
  const GridDesc& gcd = G.grids[t.grid + 1];
  const RGrid gc = rgrid(gcd);
  const int c0 = t.x0 - kRHX + 4 * lane, r0 = t.y0 - kRHY + kRR * w;
  float4* fw = fs + w * kRR * 32;  // this warp's shared rows (each thread reads only its own entries)
  RegTile x, f;
  rload(x, X + g.off, g.pitch, g.ny, c0, r0);
  if constexpr (SMF) rload_sm(fs, F + g.off, g.pitch, g.ny, c0, r0, w, lane);
  else rload(f, F + g.off, g.pitch, g.ny, c0, r0);
  const unsigned mask = rmask<FULL>(G, gd, c0, r0);
#pragma unroll
  for (int q = 0; q < kRR; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (!(mask & (1u << (q * 4 + k)))) x.v[q][k] = 0.f;
  const int gi0 = g.ox + c0, gj0 = g.oy + r0;
  const CoarseK ck = make_coarse_k<KK>(G.kap, g.problem, g.level, gi0, gj0);
  float below[4], above[4];
#pragma unroll
  for (int s = 0; s < NU; ++s) {
    exchange_rows(xbuf[0], x, below, above, w, lane);
    rhalf_sweep<KK, 0>(x, f, fw, mask, below, above, G.kap, ck, g.problem, g.level, gi0, gj0);
    exchange_rows(xbuf[1], x, below, above, w, lane);
    rhalf_sweep<KK, 1>(x, f, fw, mask, below, above, G.kap, ck, g.problem, g.level, gi0, gj0);
  }
  rstore(x, XS + g.off, g.pitch, g.ny, c0, r0, t.y0, lane);
  // residual r = f - A x (0 off the unknowns), into f's registers or shared entries; with
  // black_zero only the red nodes (the black residuals vanish after the closing black half-sweep)
  exchange_rows(xbuf[0], x, below, above, w, lane);
  const CoarseK ckr = KK == MLEV_KAPPA_PER_COARSE_CELL ? opaque(ck) : ck;
#pragma unroll
  for (int q = 0; q < kRR; ++q) {
    const float wx = __shfl_up_sync(0xffffffffu, x.v[q][3], 1);
    const float ex = __shfl_down_sync(0xffffffffu, x.v[q][0], 1);
    float fq[4];
    if constexpr (SMF) {
      const float4 fv = fw[q * 32 + lane];
      fq[0] = fv.x; fq[1] = fv.y; fq[2] = fv.z; fq[3] = fv.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) fq[k] = f.v[q][k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float xw = k == 0 ? wx : x.v[q][k == 0 ? 0 : k - 1];
      const float xe = k == 3 ? ex : x.v[q][k == 3 ? 3 : k + 1];
      const float xs = q == 0 ? below[k] : x.v[q == 0 ? 0 : q - 1][k];
      const float xn = q == kRR - 1 ? above[k] : x.v[q == kRR - 1 ? kRR - 1 : q + 1][k];
      if (black_zero && ((q + k) & 1)) {  // black: zero after the closing black half-sweep
        fq[k] = 0.f;
        continue;
      }
      float r;
      if (KK == MLEV_KAPPA_ONE) {
        r = fq[k] - (4.0f * x.v[q][k] - ((xe + xw) + (xn + xs)));
      } else {
        const EW<float> wt = rweights<KK>(G.kap, ckr, g.problem, g.level, gi0, gj0, q, k);
        r = fq[k] - (((wt.e + wt.w) + (wt.n + wt.s)) * x.v[q][k] - ((wt.e * xe + wt.w * xw) + (wt.n * xn + wt.s * xs)));
      }
      fq[k] = (mask & (1u << (q * 4 + k))) ? r : 0.f;
    }
    if constexpr (SMF) {
      fw[q * 32 + lane] = make_float4(fq[0], fq[1], fq[2], fq[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) f.v[q][k] = fq[k];
    }
  }
  // restriction: coarse node (I, J) = fine (2I, 2J) = register (q, k), q even, k in {0, 2}
  const bool out_col = lane >= 2 && lane < 30;
  float val[kRR / 2][2];
  if constexpr (SMF) {
    // from the residuals of the shared box ([64][128] floats; its outer ring reads 0, and no
    // output depends on it)
    __syncthreads();
    const float* rs = reinterpret_cast<const float*>(fs);
    auto res = [&](int R, int Cc) { return (R >= 0 && Cc >= 0) ? rs[R * kRW + Cc] : 0.f; };
#pragma unroll
    for (int q = 0; q < kRR; q += 2) {
      const int R = w * kRR + q;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int Cc = 4 * lane + 2 * kk;
        float half = res(R + 1, Cc + 1) + res(R - 1, Cc - 1);
        if (!black_zero) half += res(R, Cc + 1) + res(R, Cc - 1) + res(R + 1, Cc) + res(R - 1, Cc);
        val[q / 2][kk] = res(R, Cc) + 0.5f * half;
      }
    }
  } else {
    // needs r of the row below the warp (its q = -1) and of the column left of the lane
    exchange_rows(xbuf[1], f, below, above, w, lane);
#pragma unroll
    for (int q = 0; q < kRR; q += 2) {
      const float wr0 = __shfl_up_sync(0xffffffffu, f.v[q][3], 1);  // r(q, -1)
      const float wrm = __shfl_up_sync(0xffffffffu, q == 0 ? below[3] : f.v[q == 0 ? 0 : q - 1][3], 1);  // r(q-1, -1)
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * kk;
        const float rc = f.v[q][k];
        const float rne = f.v[q + 1][k + 1];
        const float rsw = k == 0 ? wrm : (q == 0 ? below[k - 1 < 0 ? 0 : k - 1] : f.v[q == 0 ? 0 : q - 1][k - 1 < 0 ? 0 : k - 1]);
        float half = rne + rsw;
        if (!black_zero) {
          const float re = f.v[q][k + 1];
          const float rw = k == 0 ? wr0 : f.v[q][k - 1 < 0 ? 0 : k - 1];
          const float rn = f.v[q + 1][k];
          const float rs = q == 0 ? below[k] : f.v[q == 0 ? 0 : q - 1][k];
          half += re + rw + rn + rs;
        }
        val[q / 2][kk] = rc + 0.5f * half;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kRR; q += 2) {
    const int j = r0 + q;
    if (!out_col || j < t.y0 || j >= t.y0 + kROH) continue;
    const int J = j >> 1;
    if (J > gc.ny) continue;
    const int I = c0 >> 1;
    float* fr = F + gc.off + (long long)J * gc.pitch;
    float* xr = XC + gc.off + (long long)J * gc.pitch;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int Ik = I + kk;
      if (Ik > gc.nx) continue;
      const bool u = FULL ? (Ik >= 1 && J >= 1 && Ik < gc.nx && J < gc.ny) : is_unknown(G, gcd, Ik, J);
      fr[Ik] = u ? val[q / 2][kk] : 0.f;
      xr[Ik] = 0.f;
    }
  }
}

// Up leg on one tile: x += P x_c (the coarse correction, from X on the coarser grid; with
// red_only only the red nodes, since a plain Gauss-Seidel black half-sweep opens the
// post-smoothing), then NU red-black sweeps (black first). Reads x from XS, writes X.
template <int KK, int NU, bool FULL>
__global__ void __launch_bounds__(256, KK == MLEV_KAPPA_ONE ? 2 : 3) k_rup(DevGeom G, const Tile* __restrict__ tiles,
                                                const float* __restrict__ XS, float* X, const float* __restrict__ F,
                                                int red_only) {
  __shared__ float4 xbuf[2][2][kRWarps][32];
  __shared__ float xc[34][66];  // coarse nodes [by0/2, by0/2 + 33] x [bx0/2, bx0/2 + 65]
  extern __shared__ float4 fs[];  // kappa per coarse cell: [64 rows][32 lanes], the box's f
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Tile t = tiles[blockIdx.x];
  const GridDesc& gd = G.grids[t.grid];
  const RGrid g = rgrid(gd);
  const RGrid gc = rgrid(G.grids[t.grid + 1]);
  const int bx0 = t.x0 - kRHX, by0 = t.y0 - kRHY;
  const int c0 = bx0 + 4 * lane, r0 = by0 + kRR * w;
  // coarse correction values of the box (0 outside the coarse grid)
  {
    const int CX0 = bx0 >> 1, CY0 = by0 >> 1;  // both even, so exact halves
    for (int e = threadIdx.x; e < 34 * 66; e += blockDim.x) {
      const int jj = e / 66, ii = e - jj * 66;
      const int I = CX0 + ii, J = CY0 + jj;
      float v = 0.f;
      if (I >= 0 && J >= 0 && I <= gc.nx && J <= gc.ny) v = X[gc.off + (long long)J * gc.pitch + I];
      xc[jj][ii] = v;
    }
  }
  RegTile x, f;  // f in registers for kappa = 1, in shared memory for kappa per coarse cell
  rload(x, XS + g.off, g.pitch, g.ny, c0, r0);
  if constexpr (KK == MLEV_KAPPA_PER_COARSE_CELL) rload_sm(fs, F + g.off, g.pitch, g.ny, c0, r0, w, lane);
  else rload(f, F + g.off, g.pitch, g.ny, c0, r0);
  const float4* fw = fs + w * kRR * 32;
  const unsigned mask = rmask<FULL>(G, gd, c0, r0);
  __syncthreads();
  // prolongation (exact P1 interpolation on the SW-NE mesh)
#pragma unroll
  for (int q = 0; q < kRR; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int bit = q * 4 + k;
      if (!(mask & (1u << bit))) {
        x.v[q][k] = 0.f;
        continue;
      }
      if (red_only && ((q + k) & 1)) continue;
      const int ci = 2 * lane + (k >> 1), cj = 4 * w + (q >> 1);  // coarse node (i >> 1, j >> 1) in xc
      float v;
      if (!(k & 1) && !(q & 1)) v = xc[cj][ci];
      else if ((k & 1) && !(q & 1)) v = 0.5f * (xc[cj][ci] + xc[cj][ci + 1]);
      else if (!(k & 1) && (q & 1)) v = 0.5f * (xc[cj][ci] + xc[cj + 1][ci]);
      else v = 0.5f * (xc[cj][ci] + xc[cj + 1][ci + 1]);
      x.v[q][k] += v;
    }
  const int gi0 = g.ox + c0, gj0 = g.oy + r0;
  const CoarseK ck = make_coarse_k<KK>(G.kap, g.problem, g.level, gi0, gj0);
  float below[4], above[4];
#pragma unroll
  for (int s = 0; s < NU; ++s) {  // two exchange buffers in turn: one barrier per half-sweep
    exchange_rows(xbuf[0], x, below, above, w, lane);
    rhalf_sweep<KK, 1>(x, f, fw, mask, below, above, G.kap, ck, g.problem, g.level, gi0, gj0);
    exchange_rows(xbuf[1], x, below, above, w, lane);
    rhalf_sweep<KK, 0>(x, f, fw, mask, below, above, G.kap, ck, g.problem, g.level, gi0, gj0);
  }
  rstore(x, X + g.off, g.pitch, g.ny, c0, r0, t.y0, lane);
}

// ------------------------------------------------------------------ launchers
bool rkernels_support(int kappa_kind, int level, int pre, int post, double omega) {
  return (kappa_kind == MLEV_KAPPA_ONE || (kappa_kind == MLEV_KAPPA_PER_COARSE_CELL && level >= 3)) && pre >= 1 &&
         pre <= 2 && post >= 1 && post <= 2 && omega == 1.0;
}

// dynamic shared memory of both legs: the box's f, 64 rows of 32 float4
constexpr int kRFsBytes = kRR * kRWarps * 32 * (int)sizeof(float4);

// the up leg's static buffers plus f pass the 48 KB default: raise the limit once per kernel
template <typename Kern>
static void allow_fs(Kern k, bool& done) {
  if (!done) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRFsBytes);
    done = true;
  }
}

template <int KK, int NU>
static void rdown_kk(const DevGeom& G, const Tile* tiles, int n, int full, float* X, float* XS, float* F,
                     int black_zero, cudaStream_t s) {
  constexpr int fsb = KK == MLEV_KAPPA_PER_COARSE_CELL ? kRFsBytes : 0;
  static bool a0 = false, a1 = false;
  if (full) {
    if (fsb) allow_fs(k_rdown<KK, NU, true>, a1);
    k_rdown<KK, NU, true><<<n, 256, fsb, s>>>(G, tiles, X, X, XS, F, black_zero);
  } else {
    if (fsb) allow_fs(k_rdown<KK, NU, false>, a0);
    k_rdown<KK, NU, false><<<n, 256, fsb, s>>>(G, tiles, X, X, XS, F, black_zero);
  }
}
template <int KK, int NU>
static void rup_kk(const DevGeom& G, const Tile* tiles, int n, int full, const float* XS, float* X, const float* F,
                   int red_only, cudaStream_t s) {
  constexpr int fsb = KK == MLEV_KAPPA_PER_COARSE_CELL ? kRFsBytes : 0;
  static bool a0 = false, a1 = false;
  if (full) {
    if (fsb) allow_fs(k_rup<KK, NU, true>, a1);
    k_rup<KK, NU, true><<<n, 256, fsb, s>>>(G, tiles, XS, X, F, red_only);
  } else {
    if (fsb) allow_fs(k_rup<KK, NU, false>, a0);
    k_rup<KK, NU, false><<<n, 256, fsb, s>>>(G, tiles, XS, X, F, red_only);
  }
}

void launch_rdown(const DevGeom& G, const Tile* tiles, int n, int full, float* X, float* XS, float* F, int nu,
                  int black_zero, cudaStream_t s) {
  if (!n) return;
  if (G.kap.kind == MLEV_KAPPA_ONE) {
    if (nu == 1) rdown_kk<MLEV_KAPPA_ONE, 1>(G, tiles, n, full, X, XS, F, black_zero, s);
    else rdown_kk<MLEV_KAPPA_ONE, 2>(G, tiles, n, full, X, XS, F, black_zero, s);
  } else {
    if (nu == 1) rdown_kk<MLEV_KAPPA_PER_COARSE_CELL, 1>(G, tiles, n, full, X, XS, F, black_zero, s);
    else rdown_kk<MLEV_KAPPA_PER_COARSE_CELL, 2>(G, tiles, n, full, X, XS, F, black_zero, s);
  }
}
void launch_rup(const DevGeom& G, const Tile* tiles, int n, int full, const float* XS, float* X, const float* F, int nu,
                int red_only, cudaStream_t s) {
  if (!n) return;
  if (G.kap.kind == MLEV_KAPPA_ONE) {
    if (nu == 1) rup_kk<MLEV_KAPPA_ONE, 1>(G, tiles, n, full, XS, X, F, red_only, s);
    else rup_kk<MLEV_KAPPA_ONE, 2>(G, tiles, n, full, XS, X, F, red_only, s);
  } else {
    if (nu == 1) rup_kk<MLEV_KAPPA_PER_COARSE_CELL, 1>(G, tiles, n, full, XS, X, F, red_only, s);
    else rup_kk<MLEV_KAPPA_PER_COARSE_CELL, 2>(G, tiles, n, full, XS, X, F, red_only, s);
  }
}

}  // namespace mlev
