// Device helpers shared by all kernels: unknown tests on job grids, the coefficient
// kappa on every level, and the matrix-free P1 stiffness / mass stencils on the
// SW-NE triangulation.
//
// Stencils (derived from the element matrices of Section 2.2 / Section 3 on right
// triangles with legs h): each triangle adds kappa_T / 2 to the coupling of its two
// legs and nothing to its hypotenuse, so the stiffness row is the 5-point stencil
//   (K x)_c = (wE + wW + wN + wS) x_c - wE x_E - wW x_W - wN x_N - wS x_S
// with wE = (kappa_L(c) + kappa_U(s)) / 2, wN = (kappa_U(c) + kappa_L(w)) / 2,
//      wW = (kappa_L(w) + kappa_U(sw)) / 2, wS = (kappa_U(s) + kappa_L(sw)) / 2,
// where c, s, w, sw are the cells NE, SE, NW, SW of the node; the consistent mass
// row is (h^2 / 12) (6 x_c + x_E + x_W + x_N + x_S + x_NE + x_SW).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mlev.h"
#include "mlev_internal.h"

namespace mlev {

__device__ __forceinline__ bool region_at(const DevGeom& G, const GridDesc& g, int rx, int ry) {
  return G.regions[g.roff + (long long)ry * g.rnx + rx] != 0;
}

// Node (i, j) of grid g is an unknown: strictly inside the window and all four
// adjacent cells lie in the job's region.
__device__ __forceinline__ bool is_unknown(const DevGeom& G, const GridDesc& g, int i, int j) {
  if (i < 1 || j < 1 || i >= g.nx || j >= g.ny) return false;
  if (g.full) return true;
  const int s = g.rshift;
  const int a = (i - 1) >> s, b = i >> s, c = (j - 1) >> s, d = j >> s;
  return region_at(G, g, a, c) && region_at(G, g, b, c) && region_at(G, g, a, d) && region_at(G, g, b, d);
}

// Free node (not on dOmega) of the global level-l lattice.
__device__ __forceinline__ bool is_free(const DevGeom& G, int l, int nx, int ny, int i, int j) {
  if (i < 1 || j < 1 || i >= nx || j >= ny) return false;
  if (l >= 0) {
    const int a = (i - 1) >> l, b = i >> l, c = (j - 1) >> l, d = j >> l;
    return G.cell_in[c * G.ncx + a] && G.cell_in[c * G.ncx + b] && G.cell_in[d * G.ncx + a] &&
           G.cell_in[d * G.ncx + b];
  }
  const int s = -l;  // cell (x, y) at a negative level covers coarse cell (x << s, y << s)
  const int a = (i - 1) << s, b = i << s, c = (j - 1) << s, d = j << s;
  return G.cell_in[c * G.ncx + a] && G.cell_in[c * G.ncx + b] && G.cell_in[d * G.ncx + a] &&
         G.cell_in[d * G.ncx + b];
}

__device__ __forceinline__ int lvl_cells_x(const KappaDev& kv, int l) { return l >= 0 ? kv.ncx << l : kv.ncx >> (-l); }
__device__ __forceinline__ int lvl_cells_y(const KappaDev& kv, int l) { return l >= 0 ? kv.ncy << l : kv.ncy >> (-l); }

// kappa on triangle t (0 lower, 1 upper) of cell (x, y) of level l, batch member p.
// Cells outside the lattice return 0 (they only border non-unknown nodes).
template <int KK>
__device__ __forceinline__ double kap_tri(const KappaDev& kv, int p, int l, int x, int y, int t) {
  if (KK == MLEV_KAPPA_ONE) return 1.0;
  const int nx = lvl_cells_x(kv, l), ny = lvl_cells_y(kv, l);
  if (x < 0 || y < 0 || x >= nx || y >= ny) return 0.0;
  if (KK == MLEV_KAPPA_PER_COARSE_CELL && l >= 0)
    return kv.coarse[(long long)p * kv.ncx * kv.ncy + (y >> l) * kv.ncx + (x >> l)];
  const int i = l - MLEV_LMIN;
  const double* base = kv.lvl + kv.lvl_off[i] + (long long)p * kv.lvl_bstride[i];
  return base[((long long)y * nx + x) * 2 + t];
}

struct W4 {
  double e, w, n, s;
};

// Edge weights of the stiffness row of global node (gi, gj) at level l.
template <int KK>
__device__ __forceinline__ W4 edge_weights(const KappaDev& kv, int p, int l, int gi, int gj) {
  W4 r;
  if (KK == MLEV_KAPPA_ONE) {
    r.e = r.w = r.n = r.s = 1.0;
    return r;
  }
  if (KK == MLEV_KAPPA_PER_COARSE_CELL && l >= 0) {
    // all six triangles around a node inside a coarse cell share one value
    const double* kc = kv.coarse + (long long)p * kv.ncx * kv.ncy;
    const int ci = gi >> l, cw = (gi - 1) >> l, cj = gj >> l, cs = (gj - 1) >> l;
    const double kc_c = kc[cj * kv.ncx + ci], kc_s = kc[cs * kv.ncx + ci];
    const double kc_w = kc[cj * kv.ncx + cw], kc_sw = kc[cs * kv.ncx + cw];
    r.e = 0.5 * (kc_c + kc_s);
    r.n = 0.5 * (kc_c + kc_w);
    r.w = 0.5 * (kc_w + kc_sw);
    r.s = 0.5 * (kc_s + kc_sw);
    return r;
  }
  const double kLc = kap_tri<KK>(kv, p, l, gi, gj, 0), kUc = kap_tri<KK>(kv, p, l, gi, gj, 1);
  const double kUs = kap_tri<KK>(kv, p, l, gi, gj - 1, 1);
  const double kLw = kap_tri<KK>(kv, p, l, gi - 1, gj, 0);
  const double kLsw = kap_tri<KK>(kv, p, l, gi - 1, gj - 1, 0), kUsw = kap_tri<KK>(kv, p, l, gi - 1, gj - 1, 1);
  r.e = 0.5 * (kLc + kUs);
  r.n = 0.5 * (kUc + kLw);
  r.w = 0.5 * (kLw + kUsw);
  r.s = 0.5 * (kUs + kLsw);
  return r;
}

// The same coefficient and edge weights in precision T: T = float reads the FP32 copies of
// the coefficient tables, so FP32 multigrid kernels issue no FP64 arithmetic.
template <typename T>
struct EW {
  T e, w, n, s;
};

template <typename T, int KK>
__device__ __forceinline__ T kap_tri_t(const KappaDev& kv, int p, int l, int x, int y, int t) {
  if (KK == MLEV_KAPPA_ONE) return (T)1;
  const int nx = lvl_cells_x(kv, l), ny = lvl_cells_y(kv, l);
  if (x < 0 || y < 0 || x >= nx || y >= ny) return (T)0;
  if (KK == MLEV_KAPPA_PER_COARSE_CELL && l >= 0) {
    const long long q = (long long)p * kv.ncx * kv.ncy + (y >> l) * kv.ncx + (x >> l);
    if constexpr (sizeof(T) == 4) return kv.coarse_f[q];
    else return kv.coarse[q];
  }
  const int i = l - MLEV_LMIN;
  const long long q = kv.lvl_off[i] + (long long)p * kv.lvl_bstride[i] + ((long long)y * nx + x) * 2 + t;
  if constexpr (sizeof(T) == 4) return kv.lvl_f[q];
  else return kv.lvl[q];
}

// v / d for the Gauss-Seidel update (d the stencil's diagonal): in FP32 as v times the
// correctly rounded reciprocal of d, which costs a fraction of a full-precision division (the
// result differs from v / d by at most an ulp); in FP64 the division itself.
template <typename T>
__device__ __forceinline__ T div_diag(T v, T d) {
  if constexpr (sizeof(T) == 4) return v * __frcp_rn(d);
  else return v / d;
}

template <typename T, int KK>
__device__ __forceinline__ EW<T> edge_weights_t(const KappaDev& kv, int p, int l, int gi, int gj) {
  EW<T> r;
  if (KK == MLEV_KAPPA_ONE) {
    r.e = r.w = r.n = r.s = (T)1;
    return r;
  }
  if (KK == MLEV_KAPPA_PER_COARSE_CELL && l >= 0) {
    const int ci = gi >> l, cw = (gi - 1) >> l, cj = gj >> l, cs = (gj - 1) >> l;
    const int b = p * kv.ncx * kv.ncy;  // batch x T_H cells, far below 2^31 (32-bit index math)
    T kc_c, kc_s, kc_w, kc_sw;
    if constexpr (sizeof(T) == 4) {
      kc_c = kv.coarse_f[b + cj * kv.ncx + ci];
      kc_s = kv.coarse_f[b + cs * kv.ncx + ci];
      kc_w = kv.coarse_f[b + cj * kv.ncx + cw];
      kc_sw = kv.coarse_f[b + cs * kv.ncx + cw];
    } else {
      kc_c = kv.coarse[b + cj * kv.ncx + ci];
      kc_s = kv.coarse[b + cs * kv.ncx + ci];
      kc_w = kv.coarse[b + cj * kv.ncx + cw];
      kc_sw = kv.coarse[b + cs * kv.ncx + cw];
    }
    r.e = (T)0.5 * (kc_c + kc_s);
    r.n = (T)0.5 * (kc_c + kc_w);
    r.w = (T)0.5 * (kc_w + kc_sw);
    r.s = (T)0.5 * (kc_s + kc_sw);
    return r;
  }
  const T kLc = kap_tri_t<T, KK>(kv, p, l, gi, gj, 0), kUc = kap_tri_t<T, KK>(kv, p, l, gi, gj, 1);
  const T kUs = kap_tri_t<T, KK>(kv, p, l, gi, gj - 1, 1);
  const T kLw = kap_tri_t<T, KK>(kv, p, l, gi - 1, gj, 0);
  const T kLsw = kap_tri_t<T, KK>(kv, p, l, gi - 1, gj - 1, 0), kUsw = kap_tri_t<T, KK>(kv, p, l, gi - 1, gj - 1, 1);
  r.e = (T)0.5 * (kLc + kUs);
  r.n = (T)0.5 * (kUc + kLw);
  r.w = (T)0.5 * (kLw + kUsw);
  r.s = (T)0.5 * (kUs + kLsw);
  return r;
}

// (K x)_c with the given weights (W4 or EW<T>) on a pitched array.
template <typename T, typename V, typename WW>
__device__ __forceinline__ V apply_k(const T* x, long long c, int pitch, const WW& w) {
  return (V)(w.e + w.w + w.n + w.s) * (V)x[c] - (V)w.e * (V)x[c + 1] - (V)w.w * (V)x[c - 1] -
         (V)w.n * (V)x[c + pitch] - (V)w.s * (V)x[c - pitch];
}

// (M x)_c / (h^2 / 12) on a pitched array.
template <typename T, typename V>
__device__ __forceinline__ V apply_m12(const T* x, long long c, int pitch) {
  return (V)6 * (V)x[c] + (V)x[c + 1] + (V)x[c - 1] + (V)x[c + pitch] + (V)x[c - pitch] + (V)x[c + pitch + 1] +
         (V)x[c - pitch - 1];
}

// K x and M x / (h^2 / 12) at one node for kappa = 1, sharing the sum of the four edge
// neighbours s4: K x = 4 x_c - s4, M x / (h^2 / 12) = 6 x_c + s4 + x_ne + x_sw (7 FP64
// operations for both, against 12 for apply_k and apply_m12 apart).
template <typename T, typename V>
__device__ __forceinline__ void apply_km_one(const T* x, long long c, int pitch, V& kx, V& mx) {
  const V xc = (V)x[c];
  const V s4 = ((V)x[c + 1] + (V)x[c - 1]) + ((V)x[c + pitch] + (V)x[c - pitch]);
  kx = (V)4 * xc - s4;
  mx = (V)6 * xc + s4 + ((V)x[c + pitch + 1] + (V)x[c - pitch - 1]);
}

// 2^e as a double, built from its exponent field (exact for |e| < 1023): scaling by it equals
// dividing by 2^-e bit for bit, without an FP64 division.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

__device__ __forceinline__ double level_h(double H, int l) { return H * pow2(-l); }

// Block-wide sum of NV doubles per thread into sh[0..NV-1] (deterministic tree order).
// `scratch` holds blockDim.x/32 * NV doubles. All threads must call it.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) scratch[warp * NV + k] = a;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = lane < nw ? scratch[lane * NV + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (lane == 0) out[k] = a;
    }
  }
  __syncthreads();
}

}  // namespace mlev
