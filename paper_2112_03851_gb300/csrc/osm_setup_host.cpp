// Host-side assembly of the subdomain systems of the optimized Schwarz
// method (Sec. 3) for Q2 hexahedra (Sec. 6), packed for the GPU.
//
// On an axis-aligned tensor-product mesh the Q2 stiffness and mass of any
// box of elements factor into assembled 1-D operators:
//   K_box = Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz
// with the 1-D element matrices on [0, h] (nodes 0, h/2, h)
//   K1 = 1/(3h) [[7,-8,1],[-8,16,-8],[1,-8,7]],  M1 = h/30 [[4,2,-1],[2,16,2],[-1,2,4]],
// and an interface face mass M_G = Ma (x) Mb over its two tangential
// directions.  Every matrix entry is therefore a sum of three products of
// banded 1-D entries, evaluated row by row straight into the SELL layout.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "osm_internal.h"

namespace osm {
namespace {

// Assembled 1-D Q2 operators over elements [e0, e1) of one direction.
// Node a (0 .. 2(e1-e0)) couples with a-2 .. a+2: band index a*5 + (b-a+2).
struct Band1D {
  int n = 0;
  std::vector<double> K, M, W;  // W: integral of each 1-D basis function
  void build(const std::vector<double>& c, int e0, int e1) {
    n = 2 * (e1 - e0) + 1;
    K.assign(5 * n, 0.0);
    M.assign(5 * n, 0.0);
    W.assign(n, 0.0);
    static const double k1[3][3] = {{7, -8, 1}, {-8, 16, -8}, {1, -8, 7}};
    static const double m1[3][3] = {{4, 2, -1}, {2, 16, 2}, {-1, 2, 4}};
    static const double w1[3] = {1, 4, 1};
    for (int e = e0; e < e1; ++e) {
      double h = c[e + 1] - c[e];
      int a0 = 2 * (e - e0);
      for (int a = 0; a < 3; ++a) {
        W[a0 + a] += h * w1[a] / 6.0;
        for (int b = 0; b < 3; ++b) {
          K[(a0 + a) * 5 + (b - a + 2)] += k1[a][b] / (3.0 * h);
          M[(a0 + a) * 5 + (b - a + 2)] += m1[a][b] * h / 30.0;
        }
      }
    }
  }
  double k(int a, int b) const { return K[a * 5 + (b - a + 2)]; }
  double m(int a, int b) const { return M[a * 5 + (b - a + 2)]; }
};

inline int reach(int i) { return (i % 2 == 0) ? 2 : 1; }

// Work data of one subdomain during the build.
struct SubWork {
  Band1D bx, by, bz;
  int bnx, bny, bnz;                 // box node counts
  std::vector<int32_t> box2can;      // box node -> canonical index or -1
  std::vector<int32_t> can_node;     // canonical -> full-grid node id
  std::vector<int32_t> len;          // row length per canonical index
  std::vector<int32_t> perm;         // internal row -> canonical
  std::vector<int32_t> can2int;      // canonical -> internal row
  std::vector<int32_t> slice_w;      // widths of its slices
};

}  // namespace

static bool on_boundary(const HostProblem& hp, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == hp.NX - 1 || j == hp.NY - 1 || k == hp.NZ - 1;
}

void build_load(const HostProblem& hp, const double* drho, std::vector<double>& f) {
  // f_i = 4 pi G sum_e drho_e int phi (Sec. 2) with the 1-D basis integrals
  // h (1/6, 4/6, 1/6) of each element's three nodes per direction.
  f.assign(hp.vec_rows, 0.0);
  const double four_pi_g = 4.0 * kPi * kGravity;
  static const double w1[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < hp.nsub; ++s) {
    const SubInfo& S = hp.sub[s];
    for (int ez = S.ez0; ez < S.ez1; ++ez)
      for (int ey = S.ey0; ey < S.ey1; ++ey)
        for (int ex = S.ex0; ex < S.ex1; ++ex) {
          double rho = drho[ex + (int64_t)hp.nx * (ey + (int64_t)hp.ny * ez)];
          if (rho == 0.0) continue;
          double hx = hp.xc[ex + 1] - hp.xc[ex], hy = hp.yc[ey + 1] - hp.yc[ey],
                 hz = hp.zc[ez + 1] - hp.zc[ez];
          for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
              for (int a = 0; a < 3; ++a) {
                int i = 2 * ex + a, j = 2 * ey + b, k = 2 * ez + c;
                if (on_boundary(hp, i, j, k)) continue;
                int64_t node = i + (int64_t)hp.NX * (j + (int64_t)hp.NY * k);
                int32_t row = -1;  // this subdomain's copy of the node
                for (int32_t q = hp.cp_ptr[node]; q < hp.cp_ptr[node + 1]; ++q) {
                  int32_t r = hp.cp_idx[q];
                  if (r >= S.voff && r < S.voff + S.npad) { row = r; break; }
                }
                f[row] += four_pi_g * rho * (w1[a] * hx) * (w1[b] * hy) * (w1[c] * hz);
              }
        }
  }
}

std::string build_host_problem(const osm_mesh& mesh, const double* drho, const osm_decomp& dec,
                               HostProblem& hp, bool want_fp32) {
  if (mesh.nx < 1 || mesh.ny < 1 || mesh.nz < 1) return "mesh needs at least one element per direction";
  if (!mesh.xc || !mesh.yc || !mesh.zc || !drho) return "null mesh coordinates or density";
  if (dec.sx < 1 || dec.sy < 1 || dec.sz < 1 || !dec.cx || !dec.cy || !dec.cz)
    return "bad decomposition";
  hp.nx = mesh.nx; hp.ny = mesh.ny; hp.nz = mesh.nz;
  hp.NX = 2 * hp.nx + 1; hp.NY = 2 * hp.ny + 1; hp.NZ = 2 * hp.nz + 1;
  int64_t nn = (int64_t)hp.NX * hp.NY * hp.NZ;
  if (nn >= (int64_t)1 << 31) return "node grid too large for 32-bit indices";
  hp.xc.assign(mesh.xc, mesh.xc + hp.nx + 1);
  hp.yc.assign(mesh.yc, mesh.yc + hp.ny + 1);
  hp.zc.assign(mesh.zc, mesh.zc + hp.nz + 1);
  for (auto* c : {&hp.xc, &hp.yc, &hp.zc})
    for (size_t i = 0; i + 1 < c->size(); ++i)
      if (!((*c)[i + 1] > (*c)[i]) || !std::isfinite((*c)[i + 1])) return "coordinates must increase";
  hp.sx = dec.sx; hp.sy = dec.sy; hp.sz = dec.sz;
  hp.nsub = dec.sx * dec.sy * dec.sz;
  auto check_cuts = [](const int32_t* c, int s, int n) {
    if (c[0] != 0 || c[s] != n) return false;
    for (int i = 0; i < s; ++i) if (c[i + 1] <= c[i]) return false;
    return true;
  };
  if (!check_cuts(dec.cx, dec.sx, hp.nx) || !check_cuts(dec.cy, dec.sy, hp.ny) ||
      !check_cuts(dec.cz, dec.sz, hp.nz))
    return "cuts must be strictly increasing from 0 to n";
  for (int64_t e = 0; e < (int64_t)hp.nx * hp.ny * hp.nz; ++e)
    if (!std::isfinite(drho[e])) return "density must be finite";
  hp.n_nodes = nn;
  hp.n_dofs = (int64_t)(hp.NX - 2) * (hp.NY - 2) * (hp.NZ - 2);

  const int nsub = hp.nsub;
  hp.sub.resize(nsub);
  std::vector<SubWork> W(nsub);

  // ---- pass 1: per-subdomain unknowns, row lengths, ordering, slice widths
  int bad = 0;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsub; ++s) {
    int a = s % hp.sx, b = (s / hp.sx) % hp.sy, c = s / (hp.sx * hp.sy);
    SubInfo& S = hp.sub[s];
    S.ex0 = dec.cx[a]; S.ex1 = dec.cx[a + 1];
    S.ey0 = dec.cy[b]; S.ey1 = dec.cy[b + 1];
    S.ez0 = dec.cz[c]; S.ez1 = dec.cz[c + 1];
    S.i0 = 2 * S.ex0; S.i1 = 2 * S.ex1; S.j0 = 2 * S.ey0; S.j1 = 2 * S.ey1;
    S.k0 = 2 * S.ez0; S.k1 = 2 * S.ez1;
    S.iface[0] = a > 0; S.iface[1] = a < hp.sx - 1;
    S.iface[2] = b > 0; S.iface[3] = b < hp.sy - 1;
    S.iface[4] = c > 0; S.iface[5] = c < hp.sz - 1;
    S.fmask = (S.i0 == 0 ? 1 : 0) | (S.i1 == hp.NX - 1 ? 2 : 0) | (S.j0 == 0 ? 4 : 0) |
              (S.j1 == hp.NY - 1 ? 8 : 0) | (S.k0 == 0 ? 16 : 0) | (S.k1 == hp.NZ - 1 ? 32 : 0);
    for (int f = 0; f < 6; ++f)
      if (S.iface[f]) S.fmask |= 1 << (8 + f);
    SubWork& w = W[s];
    w.bx.build(hp.xc, S.ex0, S.ex1);
    w.by.build(hp.yc, S.ey0, S.ey1);
    w.bz.build(hp.zc, S.ez0, S.ez1);
    w.bnx = S.i1 - S.i0 + 1; w.bny = S.j1 - S.j0 + 1; w.bnz = S.k1 - S.k0 + 1;
    int64_t nbox = (int64_t)w.bnx * w.bny * w.bnz;
    w.box2can.assign(nbox, -1);
    int32_t n = 0;
    for (int k = S.k0; k <= S.k1; ++k)
      for (int j = S.j0; j <= S.j1; ++j)
        for (int i = S.i0; i <= S.i1; ++i) {
          if (on_boundary(hp, i, j, k)) continue;
          w.box2can[(i - S.i0) + (int64_t)w.bnx * ((j - S.j0) + (int64_t)w.bny * (k - S.k0))] = n++;
          w.can_node.push_back(i + hp.NX * (j + hp.NY * k));
        }
    S.n = n;
    S.npad = (n + kTileRows - 1) / kTileRows * kTileRows;
    if (S.npad == 0) S.npad = kTileRows;
    auto count1d = [&](int i, int lo, int hi, int NI) {
      int cnt = 0;
      for (int ii = std::max(lo, i - reach(i)); ii <= std::min(hi, i + reach(i)); ++ii)
        if (ii > 0 && ii < NI - 1) ++cnt;
      return cnt;
    };
    w.len.resize(n);
    for (int32_t q = 0; q < n; ++q) {
      int node = w.can_node[q];
      int i = node % hp.NX, j = (node / hp.NX) % hp.NY, k = node / (hp.NX * hp.NY);
      w.len[q] = count1d(i, S.i0, S.i1, hp.NX) * count1d(j, S.j0, S.j1, hp.NY) *
                 count1d(k, S.k0, S.k1, hp.NZ);
    }
    // rows sorted by decreasing length (ties keep node order): every SELL
    // slice then holds rows of one node class and carries little padding
    w.perm.resize(n);
    std::iota(w.perm.begin(), w.perm.end(), 0);
    std::stable_sort(w.perm.begin(), w.perm.end(),
                     [&](int32_t x, int32_t y) { return w.len[x] > w.len[y]; });
    w.can2int.resize(n);
    for (int32_t r = 0; r < n; ++r) w.can2int[w.perm[r]] = r;
    int nsl = S.npad / kSliceRows;
    w.slice_w.assign(nsl, 0);
    for (int sl = 0; sl < nsl; ++sl) {
      int wmax = 0;
      for (int l = 0; l < kSliceRows; ++l) {
        int r = sl * kSliceRows + l;
        if (r < n) wmax = std::max(wmax, w.len[w.perm[r]]);
      }
      w.slice_w[sl] = (wmax + kWidthQuantum - 1) / kWidthQuantum * kWidthQuantum;
    }
    if (n < 0) bad = 1;
  }
  if (bad) return "internal error in pass 1";

  // ---- offsets
  int64_t voff = 0, coff = 0, tile = 0, slice = 0;
  hp.slice_off.clear();
  for (int s = 0; s < nsub; ++s) {
    SubInfo& S = hp.sub[s];
    S.voff = voff; S.canon_off = coff; S.tile0 = tile; S.slice0 = slice;
    voff += S.npad; coff += S.n; tile += S.npad / kTileRows; slice += S.npad / kSliceRows;
  }
  hp.vec_rows = voff; hp.n_local = coff; hp.n_tiles = tile; hp.n_slices = slice;
  if (voff >= (int64_t)1 << 31) return "problem too large for 32-bit vector indices";
  hp.slice_off.assign(hp.n_slices + 1, 0);
  {
    int64_t off = 0;
    for (int s = 0; s < nsub; ++s) {
      const SubWork& w = W[s];
      for (size_t sl = 0; sl < w.slice_w.size(); ++sl) {
        hp.slice_off[hp.sub[s].slice0 + sl] = off;
        off += (int64_t)w.slice_w[sl] * kSliceRows;
      }
    }
    hp.slice_off[hp.n_slices] = off;
    hp.sell_entries = off;
  }
  hp.cols.assign(hp.sell_entries, 0);
  hp.vals.assign(hp.sell_entries, 0.0);
  if (want_fp32) hp.vals32.assign(hp.sell_entries, 0.0f);
  else std::vector<float>().swap(hp.vals32);
  hp.tile_sub.resize(hp.n_tiles);
  for (int s = 0; s < nsub; ++s)
    for (int64_t t = 0; t < hp.sub[s].npad / kTileRows; ++t) hp.tile_sub[hp.sub[s].tile0 + t] = s;
  hp.can2vec.resize(hp.n_local);
  hp.kdiag.assign(hp.vec_rows, 0.0);
  hp.dinv0.assign(hp.vec_rows, 0.0);
  for (int s = 0; s < nsub; ++s)
    for (int32_t q = 0; q < hp.sub[s].n; ++q)
      hp.can2vec[hp.sub[s].canon_off + q] = (int32_t)(hp.sub[s].voff + W[s].can2int[q]);
  // tensor-product form (mixed handles): the 1-D bands of every subdomain and
  // the box index of every vector row
  hp.band_k.clear();
  hp.band_m.clear();
  hp.row_boxidx.clear();
  if (want_fp32) {
    hp.row_boxidx.assign(hp.vec_rows, -1);
    for (int s = 0; s < nsub; ++s) {
      SubInfo& S = hp.sub[s];
      const SubWork& w = W[s];
      S.band0 = (int32_t)(hp.band_k.size() / 5);
      for (const Band1D* b : {&w.bx, &w.by, &w.bz}) {
        hp.band_k.insert(hp.band_k.end(), b->K.begin(), b->K.end());
        hp.band_m.insert(hp.band_m.end(), b->M.begin(), b->M.end());
      }
      for (int32_t q = 0; q < S.n; ++q) {
        const int node = w.can_node[q];
        const int i = node % hp.NX, j = (node / hp.NX) % hp.NY, k = node / (hp.NX * hp.NY);
        hp.row_boxidx[S.voff + w.can2int[q]] = (i - S.i0) + w.bnx * ((j - S.j0) + w.bny * (k - S.k0));
      }
    }
  }

  // ---- pass 2: fill SELL values and the Robin (interface) entries
  struct IfaceRow {
    int32_t row;
    double mdiag;
    double tdiag[4];                  // diagonal of M_lo, M_hi, S_lo, S_hi
    std::vector<int32_t> col;
    std::vector<double> m, kv, tc;    // tc: 4 per entry (M_lo, M_hi, S_lo, S_hi)
    std::vector<int64_t> pos, pos32;
  };
  std::vector<std::vector<IfaceRow>> irows(nsub);
  // interface-column layer of K_i: (row, column, K value) of every entry whose
  // column is an interface row of the same subdomain (the stop test's K ubar)
  struct LayerRow {
    int32_t row;
    std::vector<int32_t> col;
    std::vector<double> kv;
  };
  std::vector<std::vector<LayerRow>> lrows(nsub);
  std::vector<int64_t> nnz_sub(nsub, 0);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsub; ++s) {
    const SubInfo& S = hp.sub[s];
    const SubWork& w = W[s];
    int64_t nnz = 0;
    for (int32_t r = 0; r < S.n; ++r) {
      int32_t q = w.perm[r];
      int node = w.can_node[q];
      int i = node % hp.NX, j = (node / hp.NX) % hp.NY, k = node / (hp.NX * hp.NY);
      int ai = i - S.i0, bj = j - S.j0, ck = k - S.k0;
      int64_t sl = S.slice0 + r / kSliceRows;
      int lane = r % kSliceRows;
      int64_t off = hp.slice_off[sl];
      int wdt = w.slice_w[r / kSliceRows];
      bool on_face[6] = {S.iface[0] && i == S.i0, S.iface[1] && i == S.i1,
                         S.iface[2] && j == S.j0, S.iface[3] && j == S.j1,
                         S.iface[4] && k == S.k0, S.iface[5] && k == S.k1};
      bool is_if = on_face[0] || on_face[1] || on_face[2] || on_face[3] || on_face[4] || on_face[5];
      LayerRow lr;
      lr.row = (int32_t)(S.voff + r);
      IfaceRow ir;
      if (is_if) {
        ir.row = (int32_t)(S.voff + r);
        ir.mdiag = 0.0;
        for (double& t : ir.tdiag) t = 0.0;
      }
      int jn = 0;
      for (int kk = std::max(S.k0, k - reach(k)); kk <= std::min(S.k1, k + reach(k)); ++kk)
        for (int jj = std::max(S.j0, j - reach(j)); jj <= std::min(S.j1, j + reach(j)); ++jj)
          for (int ii = std::max(S.i0, i - reach(i)); ii <= std::min(S.i1, i + reach(i)); ++ii) {
            if (on_boundary(hp, ii, jj, kk)) continue;
            int aa = ii - S.i0, bb = jj - S.j0, cc = kk - S.k0;
            double v = w.bx.k(ai, aa) * w.by.m(bj, bb) * w.bz.m(ck, cc) +
                       w.bx.m(ai, aa) * w.by.k(bj, bb) * w.bz.m(ck, cc) +
                       w.bx.m(ai, aa) * w.by.m(bj, bb) * w.bz.k(ck, cc);
            int32_t colq = w.box2can[aa + (int64_t)w.bnx * (bb + (int64_t)w.bny * cc)];
            int32_t col = w.can2int[colq];
            int64_t cpos = off + (int64_t)(jn / 4) * 128 + lane * 4 + (jn % 4);
            int64_t vpos = off + (int64_t)(jn / 2) * 64 + lane * 2 + (jn % 2);
            hp.cols[cpos] = col;
            hp.vals[vpos] = v;
            if ((S.iface[0] && ii == S.i0) || (S.iface[1] && ii == S.i1) || (S.iface[2] && jj == S.j0) ||
                (S.iface[3] && jj == S.j1) || (S.iface[4] && kk == S.k0) || (S.iface[5] && kk == S.k1)) {
              lr.col.push_back((int32_t)(S.voff + col));
              lr.kv.push_back(v);
            }
            if (want_fp32) hp.vals32[cpos] = (float)v;
            if (col == r) hp.kdiag[S.voff + r] = v;
            if (is_if) {
              // face mass (Ma (x) Mb) and tangential stiffness (Ka (x) Mb + Ma (x) Kb)
              // of every face of this subdomain holding both nodes; faces 1, 3, 5
              // (+x, +y, +z) have this subdomain on their lower side.
              double mv = 0.0, t4[4] = {0.0, 0.0, 0.0, 0.0};
              bool coupled = false;
              for (int fc = 0; fc < 6; ++fc) {
                if (!on_face[fc]) continue;
                const int ax = fc >> 1;
                const int plane = ax == 0 ? (fc & 1 ? S.i1 : S.i0) : ax == 1 ? (fc & 1 ? S.j1 : S.j0) : (fc & 1 ? S.k1 : S.k0);
                const int other = ax == 0 ? ii : ax == 1 ? jj : kk;
                if (other != plane) continue;
                coupled = true;
                double fm, fs;
                if (ax == 0) {
                  fm = w.by.m(bj, bb) * w.bz.m(ck, cc);
                  fs = w.by.k(bj, bb) * w.bz.m(ck, cc) + w.by.m(bj, bb) * w.bz.k(ck, cc);
                } else if (ax == 1) {
                  fm = w.bx.m(ai, aa) * w.bz.m(ck, cc);
                  fs = w.bx.k(ai, aa) * w.bz.m(ck, cc) + w.bx.m(ai, aa) * w.bz.k(ck, cc);
                } else {
                  fm = w.bx.m(ai, aa) * w.by.m(bj, bb);
                  fs = w.bx.k(ai, aa) * w.by.m(bj, bb) + w.bx.m(ai, aa) * w.by.k(bj, bb);
                }
                mv += fm;
                const int side = (fc & 1) ? 0 : 1;   // 0: lower side, 1: upper side
                t4[side] += fm;
                t4[2 + side] += fs;
              }
              if (coupled) {
                ir.col.push_back((int32_t)(S.voff + col));
                ir.m.push_back(mv);
                ir.kv.push_back(v);
                ir.tc.insert(ir.tc.end(), t4, t4 + 4);
                ir.pos.push_back(vpos);
                ir.pos32.push_back(cpos);
                if (col == r) {
                  ir.mdiag = mv;
                  for (int t = 0; t < 4; ++t) ir.tdiag[t] = t4[t];
                }
              }
            }
            ++jn;
          }
      // padding entries of this row: column = own row, value 0
      for (int jp = jn; jp < wdt; ++jp) {
        hp.cols[off + (int64_t)(jp / 4) * 128 + lane * 4 + (jp % 4)] = r;
        hp.vals[off + (int64_t)(jp / 2) * 64 + lane * 2 + (jp % 2)] = 0.0;
      }
      nnz += jn;
      hp.dinv0[S.voff + r] = 1.0 / hp.kdiag[S.voff + r];
      if (is_if) irows[s].push_back(std::move(ir));
      if (!lr.col.empty()) lrows[s].push_back(std::move(lr));
    }
    // padding rows of partially filled slices point at themselves
    for (int32_t r = S.n; r < S.npad; ++r) {
      int64_t off = hp.slice_off[S.slice0 + r / kSliceRows];
      int wdt = w.slice_w[r / kSliceRows];
      for (int jp = 0; jp < wdt; ++jp)
        hp.cols[off + (int64_t)(jp / 4) * 128 + (r % kSliceRows) * 4 + (jp % 4)] = r;
    }
    nnz_sub[s] = nnz;
  }
  hp.nnz = std::accumulate(nnz_sub.begin(), nnz_sub.end(), (int64_t)0);

  // ---- copies of every node (subdomain order)
  hp.cp_ptr.assign(nn + 1, 0);
  for (int s = 0; s < nsub; ++s)
    for (int32_t q = 0; q < hp.sub[s].n; ++q) hp.cp_ptr[W[s].can_node[q] + 1]++;
  for (int64_t i = 0; i < nn; ++i) hp.cp_ptr[i + 1] += hp.cp_ptr[i];
  hp.cp_idx.assign(hp.cp_ptr[nn], 0);
  {
    std::vector<int32_t> fill(hp.cp_ptr.begin(), hp.cp_ptr.end() - 1);
    for (int s = 0; s < nsub; ++s)
      for (int32_t q = 0; q < hp.sub[s].n; ++q)
        hp.cp_idx[fill[W[s].can_node[q]]++] = (int32_t)(hp.sub[s].voff + W[s].can2int[q]);
  }

  // ---- faces (canonical face layout) with their tangential 1-D masses
  hp.face_s.clear(); hp.face_t.clear(); hp.face_n.clear(); hp.face_eo.clear();
  hp.fent_face.clear(); hp.fent_row_s.clear(); hp.fent_row_t.clear();
  hp.fm_ptr.assign(1, 0); hp.fm_col.clear(); hp.fm_val.clear(); hp.fs_val.clear();
  std::vector<std::pair<int32_t, int32_t>> lam_rows;  // (vector row, lam index)
  auto add_face = [&](int s, int t, int axis, int plane, int a0, int a1, int b0, int b1) {
    const SubInfo& S = hp.sub[s];
    const SubWork& ws = W[s];
    const SubWork& wt = W[t];
    const SubInfo& T = hp.sub[t];
    // tangential 1-D masses (the face's element ranges equal the subdomain's)
    const Band1D& ba = axis == 0 ? ws.by : ws.bx;
    const Band1D& bb = axis == 2 ? ws.by : ws.bz;
    int oa = axis == 0 ? S.j0 : S.i0;
    int ob = axis == 2 ? S.j0 : S.k0;
    int na = a1 - a0 + 1, nb = b1 - b0 + 1;
    std::vector<int32_t> fmap((size_t)na * nb, -1);
    int32_t n = 0;
    auto ijk = [&](int a, int b, int& i, int& j, int& k) {
      if (axis == 0) { i = plane; j = a; k = b; }
      else if (axis == 1) { i = a; j = plane; k = b; }
      else { i = a; j = b; k = plane; }
    };
    for (int b = b0; b <= b1; ++b)
      for (int a = a0; a <= a1; ++a) {
        int i, j, k;
        ijk(a, b, i, j, k);
        if (!on_boundary(hp, i, j, k)) fmap[(a - a0) + (size_t)na * (b - b0)] = n++;
      }
    int64_t eo = hp.n_fent;
    int f = (int)hp.face_s.size();
    hp.face_s.push_back(s); hp.face_t.push_back(t); hp.face_n.push_back(n); hp.face_eo.push_back(eo);
    auto local_row = [&](const SubInfo& U, const SubWork& wu, int i, int j, int k) {
      int64_t bi = (i - U.i0) + (int64_t)wu.bnx * ((j - U.j0) + (int64_t)wu.bny * (k - U.k0));
      return (int32_t)(U.voff + wu.can2int[wu.box2can[bi]]);
    };
    for (int b = b0; b <= b1; ++b)
      for (int a = a0; a <= a1; ++a) {
        int32_t m = fmap[(a - a0) + (size_t)na * (b - b0)];
        if (m < 0) continue;
        int i, j, k;
        ijk(a, b, i, j, k);
        int32_t rs = local_row(S, ws, i, j, k), rt = local_row(T, wt, i, j, k);
        hp.fent_face.push_back(f);
        hp.fent_row_s.push_back(rs);
        hp.fent_row_t.push_back(rt);
        lam_rows.push_back({rs, (int32_t)(2 * eo + m)});
        lam_rows.push_back({rt, (int32_t)(2 * eo + n + m)});
        for (int bb2 = std::max(b0, b - reach(b)); bb2 <= std::min(b1, b + reach(b)); ++bb2)
          for (int aa2 = std::max(a0, a - reach(a)); aa2 <= std::min(a1, a + reach(a)); ++aa2) {
            int32_t m2 = fmap[(aa2 - a0) + (size_t)na * (bb2 - b0)];
            if (m2 < 0) continue;
            hp.fm_col.push_back((int32_t)(eo + m2));
            hp.fm_val.push_back(ba.m(a - oa, aa2 - oa) * bb.m(b - ob, bb2 - ob));
            hp.fs_val.push_back(ba.k(a - oa, aa2 - oa) * bb.m(b - ob, bb2 - ob) +
                                ba.m(a - oa, aa2 - oa) * bb.k(b - ob, bb2 - ob));
          }
        hp.fm_ptr.push_back((int32_t)hp.fm_col.size());
      }
    hp.n_fent += n;
  };
  hp.n_fent = 0;
  for (int c = 0; c < hp.sz; ++c)
    for (int b = 0; b < hp.sy; ++b)
      for (int a = 0; a + 1 < hp.sx; ++a) {
        int s = a + hp.sx * (b + hp.sy * c);
        add_face(s, s + 1, 0, 2 * dec.cx[a + 1], 2 * dec.cy[b], 2 * dec.cy[b + 1], 2 * dec.cz[c],
                 2 * dec.cz[c + 1]);
      }
  for (int c = 0; c < hp.sz; ++c)
    for (int b = 0; b + 1 < hp.sy; ++b)
      for (int a = 0; a < hp.sx; ++a) {
        int s = a + hp.sx * (b + hp.sy * c);
        add_face(s, s + hp.sx, 1, 2 * dec.cy[b + 1], 2 * dec.cx[a], 2 * dec.cx[a + 1], 2 * dec.cz[c],
                 2 * dec.cz[c + 1]);
      }
  for (int c = 0; c + 1 < hp.sz; ++c)
    for (int b = 0; b < hp.sy; ++b)
      for (int a = 0; a < hp.sx; ++a) {
        int s = a + hp.sx * (b + hp.sy * c);
        add_face(s, s + hp.sx * hp.sy, 2, 2 * dec.cz[c + 1], 2 * dec.cx[a], 2 * dec.cx[a + 1],
                 2 * dec.cy[b], 2 * dec.cy[b + 1]);
      }
  hp.nface = (int)hp.face_s.size();
  if ((int64_t)hp.fm_col.size() >= ((int64_t)1 << 31)) return "too many face mass entries";

  // ---- interface rows: Robin entries and received lam indices
  hp.irow.clear(); hp.irow_sub.clear(); hp.irow_mdiag.clear(); hp.irow_tdiag.clear();
  hp.im_ptr.assign(1, 0); hp.im_col.clear(); hp.im_val.clear(); hp.im_pos.clear(); hp.im_kval.clear();
  hp.im_tc.clear();
  hp.im_pos32.clear();
  std::stable_sort(lam_rows.begin(), lam_rows.end(),
                   [](const std::pair<int32_t, int32_t>& x, const std::pair<int32_t, int32_t>& y) {
                     return x.first < y.first;
                   });
  hp.ilam_ptr.assign(1, 0); hp.ilam.clear();
  size_t lp = 0;
  for (int s = 0; s < nsub; ++s) {
    auto& rows = irows[s];
    std::sort(rows.begin(), rows.end(), [](const IfaceRow& x, const IfaceRow& y) { return x.row < y.row; });
    for (auto& ir : rows) {
      hp.irow.push_back(ir.row);
      hp.irow_sub.push_back(s);
      hp.irow_mdiag.push_back(ir.mdiag);
      hp.irow_tdiag.insert(hp.irow_tdiag.end(), ir.tdiag, ir.tdiag + 4);
      hp.im_tc.insert(hp.im_tc.end(), ir.tc.begin(), ir.tc.end());
      for (size_t e = 0; e < ir.col.size(); ++e) {
        hp.im_col.push_back(ir.col[e]);
        hp.im_val.push_back(ir.m[e]);
        hp.im_pos.push_back(ir.pos[e]);
        hp.im_pos32.push_back(ir.pos32[e]);
        hp.im_kval.push_back(ir.kv[e]);
      }
      hp.im_ptr.push_back((int32_t)hp.im_col.size());
      while (lp < lam_rows.size() && lam_rows[lp].first < ir.row) ++lp;  // (never skips)
      while (lp < lam_rows.size() && lam_rows[lp].first == ir.row) hp.ilam.push_back(lam_rows[lp++].second);
      hp.ilam_ptr.push_back((int32_t)hp.ilam.size());
    }
  }
  if (hp.ilam.size() != lam_rows.size()) return "internal error: interface rows and face entries disagree";

  // ---- interface-column layer, rows in ascending order
  hp.li_row.clear(); hp.li_col.clear(); hp.li_val.clear();
  hp.li_ptr.assign(1, 0);
  for (int s = 0; s < nsub; ++s) {
    auto& rows = lrows[s];
    std::sort(rows.begin(), rows.end(), [](const LayerRow& x, const LayerRow& y) { return x.row < y.row; });
    for (const LayerRow& lr : rows) {
      hp.li_row.push_back(lr.row);
      hp.li_col.insert(hp.li_col.end(), lr.col.begin(), lr.col.end());
      hp.li_val.insert(hp.li_val.end(), lr.kv.begin(), lr.kv.end());
      if ((int64_t)hp.li_col.size() >= ((int64_t)1 << 31)) return "interface layer too large for 32-bit offsets";
      hp.li_ptr.push_back((int32_t)hp.li_col.size());
    }
  }

  // interface-row index of every layer row (every interface row is a layer
  // row: its own diagonal column is an interface column)
  {
    std::vector<int32_t> row_ir(hp.vec_rows, -1);
    for (size_t q = 0; q < hp.irow.size(); ++q) row_ir[hp.irow[q]] = (int32_t)q;
    hp.li_irow.resize(hp.li_row.size());
    size_t covered = 0;
    for (size_t k = 0; k < hp.li_row.size(); ++k) {
      hp.li_irow[k] = row_ir[hp.li_row[k]];
      covered += hp.li_irow[k] >= 0;
    }
    if (covered != hp.irow.size()) return "internal error: an interface row is missing from the layer";
  }

  // ---- load
  build_load(hp, drho, hp.f);
  single_instance_tables(hp);
  return std::string();
}

void box_cta_tables(HostProblem& hp, int zchunk) {
  const int ns = hp.nsub;
  hp.box_cta_sub.clear();
  hp.box_sub_cta0.assign(ns + 1, 0);
  int64_t ctas = 0;
  for (int s = 0; s < ns; ++s) {
    int32_t* dm = &hp.box_dims[kBoxDims * (size_t)s];
    const int bnx = dm[0], bny = dm[1], bnz = dm[2];
    const int ncb = (int)(((int64_t)bnx * bny + kTileRows - 1) / kTileRows);
    const int nch = std::max(1, (bnz + zchunk - 1) / zchunk);
    const int zc = (bnz + nch - 1) / nch;          // chunks of nearly equal length
    const int nch_used = (bnz + zc - 1) / zc;
    dm[4] = zc;
    dm[5] = ncb;
    dm[6] = nch_used;
    hp.box_sub_cta0[s] = ctas;
    for (int64_t c = 0; c < (int64_t)ncb * nch_used; ++c) hp.box_cta_sub.push_back(s);
    ctas += (int64_t)ncb * nch_used;
  }
  hp.box_sub_cta0[ns] = ctas;
  hp.box_ctas = ctas;
}

void build_box_layout(HostProblem& hp, int zchunk) {
  const int ns = hp.nsub;
  hp.box_voff.assign(ns, 0);
  hp.box_dims.assign(kBoxDims * (size_t)ns, 0);
  hp.box_tile_sub.clear();
  hp.box_sub_tile0.assign(ns + 1, 0);
  hp.box_ub_tile0.clear();
  hp.box_sub_ub0.assign(ns + 1, 0);
  hp.box_max_nx = 0;
  int64_t rows = 0, tiles = 0;
  for (int s = 0; s < ns; ++s) {
    const SubInfo& S = hp.sub[s];
    const int bnx = S.i1 - S.i0 + 1, bny = S.j1 - S.j0 + 1, bnz = S.k1 - S.k0 + 1;
    int32_t* dm = &hp.box_dims[kBoxDims * (size_t)s];
    dm[0] = bnx;
    dm[1] = bny;
    dm[2] = bnz;
    dm[3] = S.fmask;
    hp.box_max_nx = std::max(hp.box_max_nx, bnx);
    const int64_t nb = (int64_t)bnx * bny * bnz;
    const int64_t nt = std::max<int64_t>(1, (nb + kTileRows - 1) / kTileRows);
    hp.box_voff[s] = rows;
    hp.box_sub_tile0[s] = tiles;
    for (int64_t t = 0; t < nt; ++t) hp.box_tile_sub.push_back(s);
    hp.box_sub_ub0[s] = (int64_t)hp.box_ub_tile0.size();
    for (int64_t t = 0; t < nt; t += kUpdGroup) hp.box_ub_tile0.push_back(tiles + t);
    rows += nt * kTileRows;
    tiles += nt;
  }
  hp.box_sub_tile0[ns] = tiles;
  hp.box_sub_ub0[ns] = (int64_t)hp.box_ub_tile0.size();
  hp.box_rows = rows;
  hp.box_tiles = tiles;
  box_cta_tables(hp, zchunk);
  hp.row_box.assign(hp.vec_rows, -1);
  hp.box_vec.assign(hp.box_rows, -1);
  for (int64_t r = 0; r < hp.vec_rows; ++r) {
    const int32_t b = hp.row_boxidx[r];
    if (b >= 0) {
      hp.row_box[r] = (int32_t)(hp.box_voff[hp.tile_sub[r / kTileRows]] + b);
      hp.box_vec[hp.row_box[r]] = (int32_t)r;
    }
  }
}

// Residual blocks of nodes [n0, n1) of instance `inst`: about one block per
// 256 nodes (one per thread of a 256-thread block), at least one.
static void add_rblocks(HostProblem& hp, int inst, int64_t n0, int64_t n1) {
  const int64_t per = 256;
  const int64_t nb = std::max<int64_t>(1, (n1 - n0 + per - 1) / per);
  for (int64_t b = 0; b < nb; ++b) {
    hp.rblock_inst.push_back(inst);
    hp.rblock_node0.push_back(n0 + (n1 - n0) * b / nb);
  }
}

void single_instance_tables(HostProblem& hp) {
  hp.n_inst = 1;
  hp.sub_inst.assign(hp.nsub, 0);
  hp.inst_sub0 = {0, hp.nsub};
  hp.inst_node0 = {0, hp.n_nodes};
  hp.rblock_inst.clear();
  hp.rblock_node0.clear();
  add_rblocks(hp, 0, 0, hp.n_nodes);
  hp.rblock_node0.push_back(hp.n_nodes);
  hp.inst_rblock0 = {0, (int32_t)hp.rblock_inst.size()};
}

template <class T>
static void append_shift(std::vector<T>& dst, const std::vector<T>& src, T shift) {
  for (const T& v : src) dst.push_back(v + shift);
}

template <class T>
static void append(std::vector<T>& dst, const std::vector<T>& src) {
  dst.insert(dst.end(), src.begin(), src.end());
}

std::string merge_problems(std::vector<HostProblem>& parts, HostProblem& out) {
  if (parts.empty()) return "no instances";
  out = HostProblem();
  HostProblem& o = out;
  const HostProblem& first = parts[0];
  o.nx = first.nx; o.ny = first.ny; o.nz = first.nz; o.NX = first.NX; o.NY = first.NY; o.NZ = first.NZ;
  o.sx = first.sx; o.sy = first.sy; o.sz = first.sz;
  o.xc = first.xc; o.yc = first.yc; o.zc = first.zc;
  o.n_inst = (int)parts.size();
  o.inst_sub0.push_back(0);
  o.inst_node0.push_back(0);
  o.inst_rblock0.push_back(0);
  o.slice_off.clear();
  o.ilam_ptr.push_back(0);
  o.im_ptr.push_back(0);
  o.fm_ptr.push_back(0);
  o.cp_ptr.push_back(0);
  o.li_ptr.push_back(0);
  for (int i = 0; i < o.n_inst; ++i) {
    HostProblem& p = parts[i];
    const int32_t sub_off = o.nsub;
    const int64_t vec_off = o.vec_rows, tile_off = o.n_tiles, slice_off = o.n_slices, ent_off = o.sell_entries;
    const int64_t canon_off = o.n_local, node_off = o.n_nodes, fent_off = o.n_fent;
    const int32_t face_off = o.nface;
    const int64_t ilam_off = (int64_t)o.ilam.size(), im_off = (int64_t)o.im_col.size();
    const int64_t fm_off = (int64_t)o.fm_col.size(), cp_off = (int64_t)o.cp_idx.size();
    if (vec_off + p.vec_rows >= ((int64_t)1 << 31) || node_off + p.n_nodes >= ((int64_t)1 << 31) ||
        fm_off + (int64_t)p.fm_col.size() >= ((int64_t)1 << 31))
      return "batched problem too large for 32-bit indices";
    const int32_t band_off = (int32_t)(o.band_k.size() / 5);
    for (SubInfo S : p.sub) {
      S.voff += vec_off; S.canon_off += canon_off; S.tile0 += tile_off; S.slice0 += slice_off;
      S.band0 += band_off;
      o.sub.push_back(S);
    }
    append(o.band_k, p.band_k);
    append(o.band_m, p.band_m);
    append(o.row_boxidx, p.row_boxidx);
    for (int64_t k = 0; k < p.n_slices; ++k) o.slice_off.push_back(p.slice_off[k] + ent_off);
    append(o.cols, p.cols);
    append(o.vals, p.vals);
    append(o.vals32, p.vals32);
    append_shift(o.tile_sub, p.tile_sub, sub_off);
    append_shift(o.can2vec, p.can2vec, (int32_t)vec_off);
    append(o.f, p.f);
    append(o.kdiag, p.kdiag);
    append(o.dinv0, p.dinv0);
    append_shift(o.irow, p.irow, (int32_t)vec_off);
    append_shift(o.irow_sub, p.irow_sub, sub_off);
    append(o.irow_mdiag, p.irow_mdiag);
    append(o.irow_tdiag, p.irow_tdiag);
    append(o.im_tc, p.im_tc);
    for (size_t k = 1; k < p.ilam_ptr.size(); ++k) o.ilam_ptr.push_back((int32_t)(p.ilam_ptr[k] + ilam_off));
    append_shift(o.ilam, p.ilam, (int32_t)(2 * fent_off));
    for (size_t k = 1; k < p.im_ptr.size(); ++k) o.im_ptr.push_back((int32_t)(p.im_ptr[k] + im_off));
    append_shift(o.im_col, p.im_col, (int32_t)vec_off);
    append(o.im_val, p.im_val);
    append_shift(o.im_pos, p.im_pos, ent_off);
    append(o.im_kval, p.im_kval);
    append_shift(o.im_pos32, p.im_pos32, ent_off);
    append_shift(o.face_s, p.face_s, sub_off);
    append_shift(o.face_t, p.face_t, sub_off);
    append(o.face_n, p.face_n);
    append_shift(o.face_eo, p.face_eo, fent_off);
    append_shift(o.fent_face, p.fent_face, face_off);
    append_shift(o.fent_row_s, p.fent_row_s, (int32_t)vec_off);
    append_shift(o.fent_row_t, p.fent_row_t, (int32_t)vec_off);
    for (size_t k = 1; k < p.fm_ptr.size(); ++k) o.fm_ptr.push_back((int32_t)(p.fm_ptr[k] + fm_off));
    append_shift(o.fm_col, p.fm_col, (int32_t)fent_off);
    append(o.fm_val, p.fm_val);
    append(o.fs_val, p.fs_val);
    for (size_t k = 1; k < p.cp_ptr.size(); ++k) o.cp_ptr.push_back((int32_t)(p.cp_ptr[k] + cp_off));
    const int64_t li_off = (int64_t)o.li_col.size();
    if (li_off + (int64_t)p.li_col.size() >= ((int64_t)1 << 31)) return "batched interface layer too large";
    append_shift(o.li_row, p.li_row, (int32_t)vec_off);
    append_shift(o.li_col, p.li_col, (int32_t)vec_off);
    append(o.li_val, p.li_val);
    for (size_t k = 1; k < p.li_ptr.size(); ++k) o.li_ptr.push_back((int32_t)(p.li_ptr[k] + li_off));
    const int32_t irow_off = (int32_t)(o.irow.size() - p.irow.size());   // o.irow already holds this part's rows
    for (int32_t v : p.li_irow) o.li_irow.push_back(v < 0 ? -1 : v + irow_off);
    append_shift(o.cp_idx, p.cp_idx, (int32_t)vec_off);
    for (int s = 0; s < p.nsub; ++s) o.sub_inst.push_back(i);
    add_rblocks(o, i, node_off, node_off + p.n_nodes);
    o.nsub += p.nsub;
    o.vec_rows += p.vec_rows;
    o.n_tiles += p.n_tiles;
    o.n_slices += p.n_slices;
    o.sell_entries += p.sell_entries;
    o.n_local += p.n_local;
    o.n_nodes += p.n_nodes;
    o.n_dofs += p.n_dofs;
    o.nnz += p.nnz;
    o.n_fent += p.n_fent;
    o.nface += p.nface;
    o.inst_sub0.push_back(o.nsub);
    o.inst_node0.push_back(o.n_nodes);
    o.inst_rblock0.push_back((int32_t)o.rblock_inst.size());
    p = HostProblem();  // release the part
  }
  o.slice_off.push_back(o.sell_entries);
  o.rblock_node0.push_back(o.n_nodes);
  return std::string();
}

}  // namespace osm
