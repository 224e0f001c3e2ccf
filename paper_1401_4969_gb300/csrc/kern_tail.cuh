// Multigrid on grids held in shared memory by one thread block (32 x 16 threads): the
// tail of the fused V-cycle and the level-1 eigensolver's preconditioner.
#pragma once

#include "kern_common.cuh"

namespace mlev {

constexpr int kTailMaxLev = 16;

// Shared-memory grid of the tail: compact row pitch W = nx + 1, x / f values and a mask of
// the unknowns; `g` is the job's original descriptor (coordinates, level, coefficient).
template <typename T>
struct SmGrid {
  T* x;
  T* f;
  uint8_t* m;
  int nx, ny, W;
  const GridDesc* g;
};

// Red-black sweeps, the nodes of one colour spread flat over the block: slot k is row
// j = 1 + k / hw and the (k mod hw)-th node of the colour in that row (hw = nx / 2 slots per
// row, the last one empty in rows with fewer), so every lane of every warp has a node and no
// thread takes two while others idle. The nodes of a colour are independent, so the result
// does not depend on the order.
template <typename T, int KK>
__device__ void tail_smooth(const DevGeom& G, const SmGrid<T>& s, int sweeps, bool reverse, T omega) {
  const GridDesc& g = *s.g;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int hw = s.nx >> 1, slots = hw * (s.ny - 1);
  for (int it = 0; it < sweeps; ++it)
    for (int cc = 0; cc < 2; ++cc) {
      const int color = reverse ? 1 - cc : cc;
      for (int k = tid; k < slots; k += nt) {
        const int r = k / hw, j = 1 + r;
        const int i = (((color + j) & 1) ? 1 : 2) + 2 * (k - r * hw);
        if (i >= s.nx) continue;
        const int q = j * s.W + i;
        if (!s.m[q]) continue;
        const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
        const T v = s.f[q] + (T)w.e * s.x[q + 1] + (T)w.w * s.x[q - 1] + (T)w.n * s.x[q + s.W] +
                    (T)w.s * s.x[q - s.W];
        s.x[q] += omega * (div_diag<T>(v, (T)(w.e + w.w + w.n + w.s)) - s.x[q]);
      }
      __syncthreads();
    }
}

template <typename T, int KK>
__device__ __forceinline__ T tail_res(const DevGeom& G, const SmGrid<T>& s, int i, int j) {
  const int q = j * s.W + i;
  if (!s.m[q]) return (T)0;
  const GridDesc& g = *s.g;
  const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  return s.f[q] - ((T)(w.e + w.w + w.n + w.s) * s.x[q] - (T)w.e * s.x[q + 1] - (T)w.w * s.x[q - 1] -
                   (T)w.n * s.x[q + s.W] - (T)w.s * s.x[q - s.W]);
}

// f_c = P^T (f - A x)_fine, x_c = 0; black_zero as in k_restrict (pre-smoothed by plain
// Gauss-Seidel ending black: only the red nodes of the coarse hat have a residual). Coarse
// nodes flat over the block.
template <typename T, int KK>
__device__ void tail_restrict(const DevGeom& G, const SmGrid<T>& fi, const SmGrid<T>& co, bool black_zero) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int nc = co.W * (co.ny + 1);
  for (int q = tid; q < nc; q += nt) {
    co.x[q] = (T)0;
    if (!co.m[q]) continue;
    const int J = q / co.W, I = q - J * co.W;
    const int i = 2 * I, j = 2 * J;
    T half = tail_res<T, KK>(G, fi, i + 1, j + 1) + tail_res<T, KK>(G, fi, i - 1, j - 1);
    if (!black_zero)
      half += tail_res<T, KK>(G, fi, i + 1, j) + tail_res<T, KK>(G, fi, i - 1, j) +
              tail_res<T, KK>(G, fi, i, j + 1) + tail_res<T, KK>(G, fi, i, j - 1);
    co.f[q] = tail_res<T, KK>(G, fi, i, j) + (T)0.5 * half;
  }
  __syncthreads();
}

// x += P x_c; red_only as in k_prolong (the next half-sweep is black with omega = 1): then
// only the red nodes, in the flat colour slots of tail_smooth, else every interior node.
template <typename T>
__device__ void tail_prolong(const SmGrid<T>& fi, const SmGrid<T>& co, bool red_only) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int hw = red_only ? fi.nx >> 1 : fi.nx - 1, slots = hw * (fi.ny - 1);
  for (int k = tid; k < slots; k += nt) {
    const int r = k / hw, j = 1 + r;
    const int i = red_only ? ((j & 1) ? 1 : 2) + 2 * (k - r * hw) : 1 + (k - r * hw);
    if (i >= fi.nx) continue;
    const int q = j * fi.W + i;
    if (!fi.m[q]) continue;
    const int I = i >> 1, J = j >> 1, c = J * co.W + I;
    T v;
    if (!(i & 1) && !(j & 1)) v = co.x[c];
    else if ((i & 1) && !(j & 1)) v = (T)0.5 * (co.x[c] + co.x[c + 1]);
    else if (!(i & 1) && (j & 1)) v = (T)0.5 * (co.x[c] + co.x[c + co.W]);
    else v = (T)0.5 * (co.x[c] + co.x[c + co.W + 1]);
    fi.x[q] += v;
  }
  __syncthreads();
}

template <typename T>
__device__ void tail_direct(const SmGrid<T>& s, const T* __restrict__ inv, T* fbuf) {
  const int nx1 = s.nx - 1, nd = nx1 * (s.ny - 1);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int r = tid; r < nd; r += nt) {
    const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1, q = j * s.W + i;
    fbuf[r] = s.m[q] ? s.f[q] : (T)0;
  }
  __syncthreads();
  // one warp per row of the inverse: coalesced loads, shuffle reduction
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int r = warp; r < nd; r += nw) {
    T acc = (T)0;
    for (int c = lane; c < nd; c += 32) acc += inv[r * nd + c] * fbuf[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1, q = j * s.W + i;
      s.x[q] = s.m[q] ? acc : (T)0;
    }
  }
  __syncthreads();
}

// Block-wide sum over a 2-D block (linear id y * blockDim.x + x), deterministic order;
// `scratch` holds (threads / 32) * NV doubles.
template <int NV>
__device__ void block_sum_2d(double (&v)[NV], double* scratch, double* out) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
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

// The same sums with few FP64 instructions (an FP64 add holds an SM sub-partition's FP64 pipe
// for ~64 cycles, so a shuffle tree in every warp is throughput-bound): each thread stores
// its NV values to `stage` ([NV][nt] doubles), then warp w adds quantities w, w + nwarps, ...
// (nt / 32 values per lane, then one shuffle tree). All threads call it; `out` is valid after
// the return.
template <int NV>
__device__ void block_sum_t(const double (&v)[NV], double* stage, double* out) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) stage[k * nt + tid] = v[k];
  __syncthreads();
  for (int k = warp; k < NV; k += nw) {
    double a = 0.0;
    for (int q = lane; q < nt; q += 32) a += stage[k * nt + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) out[k] = a;
  }
  __syncthreads();
}

}  // namespace mlev
