// Evaluation of coarse (T_H) P1 functions at nodes of a finer level.
#pragma once

#include "kern_common.cuh"

namespace mlev {

// Value at global node (i, j) of level L of the coarse P1 function with nodal values
// c[(ncy+1)(ncx+1)] (barycentric weights in the T_H triangle containing the node).
__device__ __forceinline__ double coarse_eval(const DevGeom& G, const double* c, int L, int i, int j) {
  const int ci = min(i >> L, G.ncx - 1), cj = min(j >> L, G.ncy - 1);
  const int ri = i - (ci << L), rj = j - (cj << L);
  const double invS = pow2(-L);  // ri / 2^L exactly
  const double s = ri * invS, t = rj * invS;
  const int w = G.ncx + 1;
  const double c00 = c[cj * w + ci], c11 = c[(cj + 1) * w + ci + 1];
  if (ri >= rj) return c00 * (1.0 - s) + c[cj * w + ci + 1] * (s - t) + c11 * t;  // lower triangle
  return c00 * (1.0 - t) + c11 * s + c[(cj + 1) * w + ci] * (t - s);              // upper triangle
}

}  // namespace mlev
