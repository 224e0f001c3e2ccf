// Host planner: decomposition sets of Section 4 and the workspace layout.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mlev {

namespace {

constexpr int kTX = 32;  // node tile width used by every tiled kernel
constexpr int kTY = 8;   // node tile height
constexpr int kAlignElems = 32;

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

int pitch_for(int nodes) { return (int)round_up(nodes, kAlignElems); }

}  // namespace

// D_j must be rectangles; computes D, Omega_j (Chebyshev dilation by o_j, clipped
// to the grid and intersected with Omega) and the closed G_j as quarter-lattice
// rectangles, then labels every quarter cell.
std::string check_partition(Plan& p) {
  const int ncx = p.ncx, ncy = p.ncy;
  p.D.assign(p.m, {ncx, ncy, -1, -1});
  std::vector<int> count(p.m, 0);
  for (int cj = 0; cj < ncy; ++cj)
    for (int ci = 0; ci < ncx; ++ci) {
      int j = p.owner[cj * ncx + ci];
      bool in = p.cell_in[cj * ncx + ci] != 0;
      if (!in) {
        if (j != -1) return "cell_owner must be -1 on cells outside Omega";
        continue;
      }
      if (j < 0 || j >= p.m) return "cell_owner out of range on a cell of Omega";
      auto& r = p.D[j];
      r[0] = std::min(r[0], ci);
      r[1] = std::min(r[1], cj);
      r[2] = std::max(r[2], ci + 1);
      r[3] = std::max(r[3], cj + 1);
      count[j]++;
    }
  for (int j = 0; j < p.m; ++j) {
    auto& r = p.D[j];
    if (count[j] == 0) return "subdomain " + std::to_string(j) + " owns no cell";
    if (count[j] != (r[2] - r[0]) * (r[3] - r[1]))
      return "UNSUPPORTED: subdomain " + std::to_string(j) + " is not a rectangle of cells";
    if (p.overlap[j] < 0) return "overlap must be >= 0";
  }
  const double dq = p.delta / (0.25 * p.H);
  const int d = (int)std::lround(dq);
  if (!(p.delta > 0) || std::fabs(dq - d) > 1e-9 * std::max(1.0, dq))
    return "delta must be a positive multiple of H/4";
  auto inside = [&](int ci, int cj) {
    return ci >= 0 && cj >= 0 && ci < ncx && cj < ncy && p.cell_in[cj * ncx + ci] != 0;
  };
  p.Om.resize(p.m);
  p.G.resize(p.m);
  for (int j = 0; j < p.m; ++j) {
    auto r = p.D[j];
    int o = p.overlap[j];
    p.Om[j] = {std::max(0, r[0] - o), std::max(0, r[1] - o), std::min(ncx, r[2] + o), std::min(ncy, r[3] + o)};
    // a side of D_j is part of dD_j \ dOmega where the cell across it is in Omega
    auto side = [&](int fixed_c, int lo, int hi, bool vertical) {
      int cnt = 0;
      for (int t = lo; t < hi; ++t) cnt += vertical ? inside(fixed_c, t) : inside(t, fixed_c);
      return cnt == 0 ? 0 : (cnt == hi - lo ? 1 : -1);
    };
    int sl = side(r[0] - 1, r[1], r[3], true), sr = side(r[2], r[1], r[3], true);
    int sb = side(r[1] - 1, r[0], r[2], false), st = side(r[3], r[0], r[2], false);
    if (sl < 0 || sr < 0 || sb < 0 || st < 0)
      return "UNSUPPORTED: a side of D_" + std::to_string(j) + " is partly on dOmega";
    std::array<int, 4> g = {4 * r[0] + (sl ? d : 0), 4 * r[1] + (sb ? d : 0), 4 * r[2] - (sr ? d : 0),
                            4 * r[3] - (st ? d : 0)};
    if (g[0] >= g[2] || g[1] >= g[3]) return "delta too large: G_" + std::to_string(j) + " is empty";
    p.G[j] = g;
  }
  // quarter-cell labels
  const int qx = 4 * ncx, qy = 4 * ncy;
  p.qlabel.assign((size_t)qx * qy, 0);
  for (int y = 0; y < qy; ++y)
    for (int x = 0; x < qx; ++x) {
      int16_t lab = inside(x >> 2, y >> 2) ? 0 : -1;
      if (lab == 0)
        for (int j = 0; j < p.m; ++j) {
          const auto& g = p.G[j];
          if (x >= g[0] && x + 1 <= g[2] && y >= g[1] && y + 1 <= g[3]) {
            if (lab != 0) return "closed G_j overlap";
            lab = (int16_t)(j + 1);
          }
        }
      p.qlabel[(size_t)y * qx + x] = lab;
    }
  // closed G_j must be disjoint also on their boundaries (checked on the quarter lattice)
  for (int i = 0; i < p.m; ++i)
    for (int j = i + 1; j < p.m; ++j) {
      const auto &a = p.G[i], &b = p.G[j];
      if (a[0] <= b[2] && b[0] <= a[2] && a[1] <= b[3] && b[1] <= a[3]) return "closed G_j overlap";
    }
  return "";
}

// Host replica of the device unknown test, summed over one grid.
long long grid_unknowns(const Plan& p, const GridDesc& g) {
  if (g.full) return (long long)(g.nx - 1) * (g.ny - 1);
  long long cnt = 0;
  const uint8_t* reg = p.regions.data() + g.roff;
  const int s = g.rshift;
  for (int j = 1; j < g.ny; ++j)
    for (int i = 1; i < g.nx; ++i) {
      const int a = (i - 1) >> s, b = i >> s, c = (j - 1) >> s, d = j >> s;
      cnt += reg[c * g.rnx + a] && reg[c * g.rnx + b] && reg[d * g.rnx + a] && reg[d * g.rnx + b];
    }
  return cnt;
}

// Does the w x h block of nodes at (x0, y0) of grid g contain an unknown?
static bool block_has_unknown(const Plan& p, const GridDesc& g, int x0, int y0, int w, int h) {
  const int xa = std::max(1, x0), xb = std::min(g.nx - 1, x0 + w - 1);
  const int ya = std::max(1, y0), yb = std::min(g.ny - 1, y0 + h - 1);
  if (xa > xb || ya > yb) return false;
  if (g.full) return true;
  const uint8_t* reg = p.regions.data() + g.roff;
  const int s = g.rshift;
  for (int j = ya; j <= yb; ++j)
    for (int i = xa; i <= xb; ++i) {
      const int a = (i - 1) >> s, b = i >> s, c = (j - 1) >> s, d = j >> s;
      if (reg[c * g.rnx + a] && reg[c * g.rnx + b] && reg[d * g.rnx + a] && reg[d * g.rnx + b]) return true;
    }
  return false;
}

std::string Plan::build(const mlev_opts& o) {
  if (!ready()) return "STATE: set domain, partition, levels and forms before solving";
  tsize = o.precision == MLEV_PREC_FP64 ? 8 : 4;
  tail_nodes = o.tail_nodes;
  std::string err = check_partition(*this);
  if (!err.empty()) return err;

  // ---- level-1 hierarchy depth: coarsen T_H while the cell mask stays block-aligned ----
  l1_lc = 0;
  for (int s = 1; s <= -MLEV_LMIN; ++s) {
    int b = 1 << s;
    if (ncx % b || ncy % b || ncx / b < 2 || ncy / b < 2) break;
    bool ok = true;
    for (int cj = 0; cj < ncy && ok; ++cj)
      for (int ci = 0; ci < ncx && ok; ++ci)
        ok = cell_in[cj * ncx + ci] == cell_in[(cj & ~(b - 1)) * ncx + (ci & ~(b - 1))];
    if (!ok) break;
    // the coarsest grid must keep at least one unknown
    int cx = ncx / b, cy = ncy / b, unk = 0;
    for (int y = 1; y < cy; ++y)
      for (int x = 1; x < cx; ++x) {
        bool all = true;
        for (int dy = -1; dy <= 0; ++dy)
          for (int dx = -1; dx <= 0; ++dx) all = all && cell_in[((y + dy) * b) * ncx + (x + dx) * b];
        unk += all;
      }
    if (!unk) break;
    l1_lc = -s;
  }

  // ---- global layout ----
  std::memset(&glay, 0, sizeof(glay));
  for (int l = l1_lc; l <= n; ++l) {
    int i = l - MLEV_LMIN;
    glay.nx[i] = l >= 0 ? ncx << l : ncx >> (-l);
    glay.ny[i] = l >= 0 ? ncy << l : ncy >> (-l);
    glay.pitch[i] = pitch_for(glay.nx[i] + 1);
  }
  glay.bstride = round_up((long long)(lvl_ny(n) + 1) * lvl_pitch(n), 64);
  {
    long long nf = 0;
    const int nxn = lvl_nx(n), nyn = lvl_ny(n), s = n;
    for (int y = 1; y < nyn; ++y)
      for (int x = 1; x < nxn; ++x) {
        bool all = true;
        for (int dy = -1; dy <= 0 && all; ++dy)
          for (int dx = -1; dx <= 0 && all; ++dx) all = cell_in[((y + dy) >> s) * ncx + ((x + dx) >> s)] != 0;
        nf += all;
      }
    n_fine = nf;
    int nc = 0;
    for (int y = 1; y < ncy; ++y)
      for (int x = 1; x < ncx; ++x)
        nc += cell_in[y * ncx + x] && cell_in[(y - 1) * ncx + x] && cell_in[y * ncx + x - 1] &&
              cell_in[(y - 1) * ncx + x - 1];
    n_coarse = nc;
  }
  nhb = (ncx - 1) * (ncy - 1);
  bw = ncx;
  nd_max = 0;
  for (int j = 0; j < m; ++j) nd_max = std::max(nd_max, (Om[j][2] - Om[j][0] - 1) * (Om[j][3] - Om[j][1] - 1));
  nd_max = std::max(nd_max, 1);
  sub_direct = nd_max <= kDirectMax;

  // ---- region grids ----
  regions.clear();
  auto add_region = [&](const std::vector<uint8_t>& r) {
    long long off = (long long)regions.size();
    regions.insert(regions.end(), r.begin(), r.end());
    while (regions.size() % 16) regions.push_back(0);
    return off;
  };
  std::vector<long long> sub_roff(m);
  std::vector<int> sub_full(m);
  for (int j = 0; j < m; ++j) {
    const auto& r = Om[j];
    std::vector<uint8_t> reg;
    bool full = true;
    for (int cj = r[1]; cj < r[3]; ++cj)
      for (int ci = r[0]; ci < r[2]; ++ci) {
        reg.push_back(cell_in[cj * ncx + ci] ? 1 : 0);
        full = full && cell_in[cj * ncx + ci];
      }
    sub_roff[j] = add_region(reg);
    sub_full[j] = full;
  }
  // G_{m+1} region: quarter cells (level 2) with label 0; when it is a union of level-1 cells
  // (delta a multiple of H/2) the strip hierarchy coarsens one level further, to T_{h_1}
  std::vector<uint8_t> sreg(qlabel.size());
  for (size_t i = 0; i < qlabel.size(); ++i) sreg[i] = qlabel[i] == 0;
  strip_lvl = 1;
  for (int y = 0; y < 2 * ncy && strip_lvl == 1; ++y)
    for (int x = 0; x < 2 * ncx && strip_lvl == 1; ++x) {
      const int q = (2 * y) * (4 * ncx) + 2 * x;
      const uint8_t v = sreg[q];
      if (sreg[q + 1] != v || sreg[q + 4 * ncx] != v || sreg[q + 4 * ncx + 1] != v) strip_lvl = 2;
    }
  if (strip_lvl == 1) {
    std::vector<uint8_t> s1((size_t)4 * ncx * ncy);
    for (int y = 0; y < 2 * ncy; ++y)
      for (int x = 0; x < 2 * ncx; ++x) s1[y * 2 * ncx + x] = sreg[(2 * y) * (4 * ncx) + 2 * x];
    sreg.swap(s1);
  }
  strip_coarse_nodes = ((ncx << strip_lvl) + 1) * ((ncy << strip_lvl) + 1);
  const long long strip_roff = add_region(sreg);
  std::vector<uint8_t> l1reg;
  {
    int b = 1 << (-l1_lc);
    for (int y = 0; y < ncy / b; ++y)
      for (int x = 0; x < ncx / b; ++x) l1reg.push_back(cell_in[(y * b) * ncx + x * b] ? 1 : 0);
  }
  const long long l1_roff = add_region(l1reg);
  bool dom_full = true;
  for (auto c : cell_in) dom_full = dom_full && c;

  // ---- grids and tiles ----
  n_tmap_grids = 0;
  grids.clear();
  tiles.clear();
  sub_top.clear();
  lp.assign(n + 1, LevelPlan());
  std::vector<long long> gunk;  // unknowns per grid
  auto add_tiles_for = [&](int gi) {
    const GridDesc& g = grids[gi];
    for (int y = 0; y <= g.ny; y += kTY)
      for (int x = 0; x <= g.nx; x += kTX) tiles.push_back(Tile{gi, x, y});
  };
  auto unk_of = [&](int gi) {
    while ((int)gunk.size() <= gi) gunk.push_back(-1);
    if (gunk[gi] < 0) gunk[gi] = grid_unknowns(*this, grids[gi]);
    return gunk[gi];
  };
  for (int L = 2; L <= n; ++L) {
    LevelPlan& P = lp[L];
    P.grid_begin = (int)grids.size();
    long long pool = 0, pool64 = 0;
    const int sdmax = L - strip_lvl;  // strip depths 0 .. sdmax (coarsest grid on level strip_lvl)
    std::vector<std::vector<int>> sub_by_depth(L + 1), strip_by_depth(sdmax + 1);
    std::vector<int> sub_coarse, sub_topg, strip_coarse;
    P.sub_top_off = (int)sub_top.size();
    sub_top.resize(sub_top.size() + (size_t)B * m);
    for (int b = 0; b < B; ++b) {
      for (int j = 0; j < m; ++j) {
        const auto& r = Om[j];
        int job = b * m + j;
        for (int dpt = 0; dpt <= L; ++dpt) {
          int l = L - dpt;
          GridDesc g{};
          g.nx = (r[2] - r[0]) << l;
          g.ny = (r[3] - r[1]) << l;
          g.pitch = pitch_for(g.nx + 1);
          g.ox = r[0] << l;
          g.oy = r[1] << l;
          g.level = l;
          g.problem = b;
          g.full = sub_full[j];
          g.rshift = l;
          g.rnx = r[2] - r[0];
          g.rny = r[3] - r[1];
          g.job = job;
          g.depth = dpt;
          g.roff = sub_roff[j];
          g.off = pool;
          pool += round_up((long long)(g.ny + 1) * g.pitch, kAlignElems);
          g.off64 = -1;
          g.tmap = -1;
          if (dpt == 0) {
            g.off64 = pool64;
            pool64 += round_up((long long)(g.ny + 1) * g.pitch, kAlignElems);
          }
          int gi = (int)grids.size();
          grids.push_back(g);
          sub_by_depth[dpt].push_back(gi);
          if (dpt == 0) {
            sub_topg.push_back(gi);
            sub_top[P.sub_top_off + job] = gi;
          }
          if (dpt == L) sub_coarse.push_back(gi);
        }
      }
      for (int dpt = 0; dpt <= sdmax; ++dpt) {
        int l = L - dpt;
        GridDesc g{};
        g.nx = ncx << l;
        g.ny = ncy << l;
        g.pitch = pitch_for(g.nx + 1);
        g.ox = 0;
        g.oy = 0;
        g.level = l;
        g.problem = b;
        g.full = 0;
        g.rshift = l - strip_lvl;
        g.rnx = ncx << strip_lvl;
        g.rny = ncy << strip_lvl;
        g.job = B * m + b;
        g.depth = dpt;
        g.roff = strip_roff;
        g.off = pool;
        pool += round_up((long long)(g.ny + 1) * g.pitch, kAlignElems);
        g.off64 = -1;
        g.tmap = -1;
        if (dpt == 0) {
          g.off64 = pool64;
          pool64 += round_up((long long)(g.ny + 1) * g.pitch, kAlignElems);
        }
        int gi = (int)grids.size();
        grids.push_back(g);
        strip_by_depth[dpt].push_back(gi);
        if (dpt == sdmax) strip_coarse.push_back(gi);
      }
    }
    P.grid_end = (int)grids.size();
    P.sub.resize(L + 1);
    for (int dpt = 0; dpt <= L; ++dpt) {
      P.sub[dpt].off = (long long)tiles.size();
      for (int gi : sub_by_depth[dpt]) {
        add_tiles_for(gi);
        P.sub[dpt].unk += unk_of(gi);
      }
      P.sub[dpt].count = (int)((long long)tiles.size() - P.sub[dpt].off);
    }
    P.strip.resize(sdmax + 1);
    for (int dpt = 0; dpt <= sdmax; ++dpt) {
      P.strip[dpt].off = (long long)tiles.size();
      for (int gi : strip_by_depth[dpt]) {
        add_tiles_for(gi);
        P.strip[dpt].unk += unk_of(gi);
      }
      P.strip[dpt].count = (int)((long long)tiles.size() - P.strip[dpt].off);
    }
    auto list_of = [&](const std::vector<int>& gl) {
      TileList t;
      t.off = (long long)tiles.size();
      for (int gi : gl) {
        tiles.push_back(Tile{gi, 0, 0});
        t.unk += unk_of(gi);
      }
      t.count = (int)gl.size();
      return t;
    };
    P.sub_coarsest = list_of(sub_coarse);
    P.sub_top = list_of(sub_topg);
    P.strip_coarsest = list_of(strip_coarse);
    // ---- fused multigrid: tail depth and tile lists
    auto tail_bytes = [&](int gi, int nlev, int extra) {
      long long tot = 0;
      for (int k = 0; k < nlev; ++k) {
        const GridDesc& g = grids[gi + k];
        tot += (long long)(g.nx + 1) * (g.ny + 1);
        tot = (tot + 1) & ~1LL;
      }
      return (size_t)(2 * tot + extra) * tsize + (size_t)tot;  // x, f, dense-solve buffer, unknown mask
    };
    auto plan_fused = [&](const std::vector<std::vector<int>>& by_depth, std::vector<TileList>& fl, int& dt,
                          TileList& tail, size_t& tail_smem, int extra, std::vector<TileList>& rl,
                          std::vector<int>& rfull) {
      const int D = (int)by_depth.size() - 1;
      dt = D + 1;
      tail_smem = 0;
      for (int d = 0; d <= D; ++d) {
        size_t need = 0;
        long long nodes = 0;
        for (int gi : by_depth[d]) {
          need = std::max(need, tail_bytes(gi, D - d + 1, extra));
          nodes = std::max(nodes, (long long)(grids[gi].nx + 1) * (grids[gi].ny + 1));
        }
        // the tail is one block per job: cap its first grid so the larger grids keep the
        // tiled (many-block) kernels; the coarsest grid always goes to the tail
        if (need <= kTailBudget && (tail_nodes <= 0 || nodes <= tail_nodes || d == D)) {
          dt = d;
          tail_smem = need;
          break;
        }
      }
      fl.assign(std::min(dt, D + 1), TileList());
      for (int d = 0; d < (int)fl.size(); ++d) {
        fl[d].off = (long long)tiles.size();
        for (int gi : by_depth[d]) {
          const GridDesc& g = grids[gi];
          for (int y = 0; y <= g.ny; y += kFusedTile)
            for (int x = 0; x <= g.nx; x += kFusedTile)
              if (block_has_unknown(*this, g, x, y, kFusedTile, kFusedTile)) tiles.push_back(Tile{gi, x, y});
          fl[d].unk += unk_of(gi);
        }
        fl[d].count = (int)((long long)tiles.size() - fl[d].off);
      }
      rl.assign(fl.size(), TileList());
      rfull.assign(fl.size(), 1);
      for (int d = 0; d < (int)rl.size(); ++d) {
        rl[d].off = (long long)tiles.size();
        for (int gi : by_depth[d]) {
          const GridDesc& g = grids[gi];
          rfull[d] = rfull[d] && g.full;
          for (int y = 0; y <= g.ny; y += MLEV_RTILE_H)
            for (int x = 0; x <= g.nx; x += MLEV_RTILE_W)
              if (block_has_unknown(*this, g, x, y, MLEV_RTILE_W, MLEV_RTILE_H)) tiles.push_back(Tile{gi, x, y});
          rl[d].unk += unk_of(gi);
        }
        rl[d].count = (int)((long long)tiles.size() - rl[d].off);
      }
      if (dt <= D) {
        tail.off = (long long)tiles.size();
        for (int gi : by_depth[dt]) {
          tiles.push_back(Tile{gi, 0, 0});
          tail.unk += unk_of(gi);
        }
        tail.count = (int)by_depth[dt].size();
      }
    };
    plan_fused(sub_by_depth, P.sub_f, P.sub_dt, P.sub_tail, P.sub_tail_smem, sub_direct ? nd_max : 0, P.sub_r,
               P.sub_r_full);
    plan_fused(strip_by_depth, P.strip_f, P.strip_dt, P.strip_tail, P.strip_tail_smem, 0, P.strip_r,
               P.strip_r_full);
    // TMA tensor maps for every grid a fused down / up kernel reads (depths 0 .. dt)
    auto give_maps = [&](const std::vector<std::vector<int>>& by_depth, int dt) {
      if (dt == 0) return;
      for (int d = 0; d <= std::min(dt, (int)by_depth.size() - 1); ++d)
        for (int gi : by_depth[d]) grids[gi].tmap = 3 * n_tmap_grids++;
    };
    give_maps(sub_by_depth, P.sub_dt);
    give_maps(strip_by_depth, P.strip_dt);
    P.pool_elems = pool;
    P.pool64_elems = pool64;
    // unknown counts per problem (reports and the traffic model)
    P.n_local = P.sub[0].unk / B;
    P.n_strip = P.strip[0].unk / B;
    {
      long long nf = 0;
      const int nxl = ncx << L, nyl = ncy << L;
      for (int y = 1; y < nyl; ++y)
        for (int x = 1; x < nxl; ++x) {
          bool all = true;
          for (int dy = -1; dy <= 0 && all; ++dy)
            for (int dx = -1; dx <= 0 && all; ++dx) all = cell_in[((y + dy) >> L) * ncx + ((x + dx) >> L)] != 0;
          nf += all;
        }
      P.n_free = nf;
    }
  }
  // level-1 job grids (one job per problem), levels 1 .. l1_lc
  l1_grid_begin = (int)grids.size();
  l1_nlev = 1 - l1_lc + 1;
  long long l1pool = 0;
  for (int b = 0; b < B; ++b)
    for (int dpt = 0; dpt < l1_nlev; ++dpt) {
      int l = 1 - dpt;
      GridDesc g{};
      g.nx = lvl_nx(l);
      g.ny = lvl_ny(l);
      g.pitch = lvl_pitch(l);
      g.level = l;
      g.problem = b;
      g.full = dom_full;
      g.rshift = l - l1_lc;
      g.rnx = lvl_nx(l1_lc);
      g.rny = lvl_ny(l1_lc);
      g.job = -1 - b;
      g.depth = dpt;
      g.roff = l1_roff;
      g.off = l1pool;
      l1pool += round_up((long long)(g.ny + 1) * g.pitch, kAlignElems);
      g.off64 = -1;
      g.tmap = -1;
      grids.push_back(g);
    }
  l1_pool_elems = l1pool;

  // ---- workspace layout ----
  size_t cur = 0;
  auto take = [&](Span& s, size_t bytes) {
    s.off = cur;
    s.bytes = bytes;
    cur += (bytes + 255) / 256 * 256;
  };
  take(w_grids, grids.size() * sizeof(GridDesc));
  take(w_tiles, std::max<size_t>(1, tiles.size()) * sizeof(Tile));
  take(w_regions, std::max<size_t>(16, regions.size()));
  take(w_qlabel, qlabel.size() * sizeof(int16_t));
  take(w_cellin, cell_in.size());
  take(w_subtop, std::max<size_t>(1, sub_top.size()) * sizeof(int));
  take(w_tmaps, std::max<size_t>(1, (size_t)3 * n_tmap_grids) * MLEV_TMAP_BYTES);
  tables_bytes = cur;
  // coefficient staging and per-level triangle values
  size_t kst = 0;
  if (kappa_kind == MLEV_KAPPA_PER_COARSE_CELL) kst = (size_t)B * ncx * ncy;
  if (kappa_kind == MLEV_KAPPA_PER_FINE_ELEM) kst = (size_t)B * lvl_nx(n) * lvl_ny(n) * 2;
  take(w_kstage, kst * 8);
  std::memset(&kap_template, 0, sizeof(kap_template));
  kap_template.kind = kappa_kind;
  kap_template.ncx = ncx;
  kap_template.ncy = ncy;
  long long klv = 0;
  for (int l = l1_lc; l <= n; ++l) {
    bool need = (kappa_kind == MLEV_KAPPA_PER_FINE_ELEM) || (kappa_kind == MLEV_KAPPA_PER_COARSE_CELL && l < 0);
    int i = l - MLEV_LMIN;
    kap_template.lvl_off[i] = klv;
    kap_template.lvl_bstride[i] = (long long)lvl_nx(l) * lvl_ny(l) * 2;
    if (need) klv += (long long)B * lvl_nx(l) * lvl_ny(l) * 2;
  }
  take(w_klvl, (size_t)std::max<long long>(klv, 1) * 8);
  take(w_klvl_f, (size_t)std::max<long long>(klv, 1) * 4);  // FP32 copies for the FP32 multigrid
  take(w_kcf, kappa_kind == MLEV_KAPPA_PER_COARSE_CELL ? (size_t)B * ncx * ncy * 4 : 0);
  take(w_band, (size_t)2 * B * nhb * (bw + 1) * 8);
  const size_t gbytes = (size_t)B * glay.bstride * 8;
  take(w_ut[0], gbytes);
  take(w_ut[1], gbytes);
  take(w_uin, gbytes);
  take(w_r, gbytes);
  const size_t l1bytes = (size_t)B * round_up((long long)(lvl_ny(1) + 1) * lvl_pitch(1), 64) * 8;
  take(w_l1vec, 10 * l1bytes);
  take(w_l1pool[0], (size_t)l1_pool_elems * tsize);
  take(w_l1pool[1], (size_t)l1_pool_elems * tsize);
  long long pmax = 0, p64max = 0;
  for (int L = 2; L <= n; ++L) {
    pmax = std::max(pmax, lp[L].pool_elems);
    p64max = std::max(p64max, lp[L].pool64_elems);
  }
  take(w_x, (size_t)pmax * tsize);
  take(w_f, (size_t)pmax * tsize);
  take(w_x64, (size_t)p64max * 8);
  take(w_xs, tsize == 4 ? (size_t)pmax * 4 : 0);
  take(w_aug, (size_t)B * ncx * ncy * 12 * 8);
  take(w_lam, (size_t)B * (n + 1) * 8);
  take(w_c, (size_t)B * (ncx + 1) * (ncy + 1) * 8);
  take(w_c0, (size_t)B * 8);
  take(w_stat, (size_t)B * mlev_stat_stride(n) * 8);
  take(w_jobnorm, (size_t)B * (m + 1) * 2 * 8);
  take(w_chol, (size_t)B * ((size_t)nhb * (bw + 1) + 5 * (size_t)nhb) * 8);
  take(w_rrpre, tsize == 4 ? (size_t)B * mlev_rr_prefactor_stride(nhb, bw) : 0);
  take(w_out_lam, (size_t)B * 8);
  take(w_out_u, (size_t)B * (lvl_nx(n) + 1) * (lvl_ny(n) + 1) * 8);
  take(w_cinv, sub_direct ? (size_t)B * m * nd_max * nd_max * tsize : 0);
  // ---- several eigenpairs
  msub = 0;
  m_nb1 = 0;
  if (q > 1) {
    if (q > MLEV_MAX_EIGENPAIRS) return "q exceeds MLEV_MAX_EIGENPAIRS";
    if (kappa_on_device) return "UNSUPPORTED: several eigenpairs need the coefficient given on the host";
    const int nx1 = lvl_nx(1), ny1 = lvl_ny(1);
    m_nb1 = (nx1 - 1) * (ny1 - 1);
    msub = std::min(16, q + 4);
    if (nx1 - 1 > 31 || ncx - 1 > 31)
      return "UNSUPPORTED: several eigenpairs need at most 16 coarse cells per side";
    if (sub_eig_smem_bytes(m_nb1, nx1 - 1, msub) > (size_t)MLEV_SUBEIG_SMEM_MAX ||
        sub_eig_smem_bytes(nhb, bw - 1, msub) > (size_t)MLEV_SUBEIG_SMEM_MAX)
      return "UNSUPPORTED: the level-1 band factor of several eigenpairs does not fit in shared memory";
    const size_t Nmax = (size_t)std::max(m_nb1, nhb + q);
    const size_t band1 = (size_t)Breal * m_nb1 * (nx1 + 1) * 8;
    take(w_mk1, band1);
    take(w_mm1, band1);
    const size_t blk = (size_t)Breal * msub * Nmax * 8;
    take(w_mX, blk);
    take(w_mY, blk);
    take(w_mAY, blk);
    take(w_mBY, blk);
    take(w_mZ, (size_t)Breal * q * nhb * 8);
    take(w_mGa, (size_t)Breal * q * nhb * 8);
    take(w_mGb, (size_t)Breal * q * nhb * 8);
    take(w_mAq, (size_t)Breal * q * q * 8);
    take(w_mBq, (size_t)Breal * q * q * 8);
    take(w_mD, (size_t)Breal * q * q * 8);
    take(w_mth, (size_t)Breal * msub * 8);
    take(w_mcross, (size_t)Breal * ncx * ncy * (q * (q + 1) / 2) * 2 * 8);
  }
  ws_bytes = cur;
  // ---- adjoint regions (only mlev_grad_kappa touches them) ----
  const size_t ncoef = (size_t)(ncx + 1) * (ncy + 1);
  take(g_ck_ut, (size_t)n * gbytes);                // u~_k of levels 1..n
  take(g_ck_c, (size_t)(n + 1) * B * ncoef * 8);    // coarse coefficients of u_{h_k}, k = 0..n
  take(g_ck_c0, (size_t)(n + 1) * B * 8);
  take(g_ubar[0], gbytes);
  take(g_ubar[1], gbytes);
  take(g_utbar, gbytes);
  take(g_sbar, gbytes);
  take(g_rbar, gbytes);
  take(g_tbuf, tsize == 4 ? (size_t)p64max * 8 : (size_t)pmax * 8);
  long long glacc = 0;
  for (int l = 1; l <= n; ++l) {
    gl_off[l] = glacc;
    glacc += (long long)B * lvl_nx(l) * lvl_ny(l) * 2;
  }
  take(g_gl, (size_t)glacc * 8);
  take(g_coef, (size_t)B * (3 * ncoef + 8) * 8);
  take(g_part2, (size_t)B * ncx * ncy * 5 * 8);
  adj_nblk = ((lvl_nx(n) + 1 + 31) / 32) * ((lvl_ny(n) + 1 + 7) / 8);
  take(g_lbpart, (size_t)B * adj_nblk * 8);
  take(g_lambar, (size_t)B * (n + 1) * 8);
  take(g_rrscr, (size_t)B * ((size_t)nhb * (bw + 1) + 10 * (size_t)nhb) * 8);
  ws_grad_bytes = cur;
  return "";
}

}  // namespace mlev
