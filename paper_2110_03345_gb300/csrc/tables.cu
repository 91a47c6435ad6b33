// Interpolation and injection tables of off-grid sources and receivers
// (Sec. 2.4: bi-/tri-linear interpolation; Kaiser-windowed sinc weights on
// request), bucketed by kernel tile so that every node is updated by the
// thread that owns it.
#include "fwi_plan.cuh"

namespace fwi {

namespace {
constexpr double kPiD = 3.14159265358979323846;
}  // namespace

Corners point_corners(const fwi_plan* P, const double* xyz) {
  // xyz in axis order slowest first; map to (x, y, z)
  const int nd = P->grid.ndim;
  double c3[3] = {0, 0, 0};
  for (int d = 0; d < nd; ++d) c3[nd - 1 - d] = xyz[d];
  int base[3] = {0, 0, 0};
  double f[3] = {0, 0, 0};
  for (int a = 0; a < nd; ++a) {
    const double xi = c3[a] / P->h[a];
    int i0 = (int)std::floor(xi);
    i0 = std::min(std::max(i0, 0), P->n3[a] - 2);
    base[a] = i0;
    f[a] = xi - (double)i0;
  }
  Corners C{};
  C.n = 1 << nd;
  for (int c = 0; c < C.n; ++c) {
    double w = 1.0;
    for (int a = 0; a < 3; ++a) {
      const int up = (a < nd) ? ((c >> a) & 1) : 0;
      C.node[c][a] = base[a] + up;
      if (a < nd) w *= up ? f[a] : (1.0 - f[a]);
    }
    C.w[c] = w;
  }
  return C;
}

long long node_index(const Layout& L, const int* n) { return L.index(n[2], n[1], n[0]); }

int interp_nodes(int interp, int ndim) {
  if (interp == FWI_INTERP_SINC) {
    int n = 1;
    for (int d = 0; d < ndim; ++d) n *= 2 * FWI_SINC_RADIUS;
    return n;
  }
  return 1 << ndim;
}

// Kaiser-windowed sinc along one axis: the 2r nodes floor(x)-r+1 .. floor(x)+r
// with w = I0(b sqrt(1 - (d/r)^2)) / I0(b) * sin(pi d) / (pi d), d = node - x.
bool sinc_axis(double x, long long n, int* first, double* w) {
  constexpr int r = FWI_SINC_RADIUS;
  constexpr double b = FWI_SINC_KAISER_B;
  auto bessel_i0 = [](double v) {          // power series sum_k ((v/2)^k / k!)^2
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200 && term > 1e-18 * sum; ++k) {
      term *= (v / (2.0 * k)) * (v / (2.0 * k));
      sum += term;
    }
    return sum;
  };
  const long long f = (long long)std::floor(x);
  if (f - r + 1 < 0 || f + r > n - 1) return false;
  const double i0b = bessel_i0(b);
  *first = (int)(f - r + 1);
  for (int j = 0; j < 2 * r; ++j) {
    const double dd = (double)(*first + j) - x;
    const double q = 1.0 - (dd / r) * (dd / r);
    const double win = std::fabs(dd) <= r ? bessel_i0(b * std::sqrt(q > 0.0 ? q : 0.0)) / i0b : 0.0;
    const double sn = dd == 0.0 ? 1.0 : std::sin(kPiD * dd) / (kPiD * dd);
    w[j] = win * sn;
  }
  return true;
}

bool point_stencil(const fwi_plan* P, const double* xyz, PointSt& out) {
  const int nd = P->grid.ndim;
  if (P->opt.interp != FWI_INTERP_SINC) {
    const Corners C = point_corners(P, xyz);
    out.n = C.n;
    out.node.resize(3 * C.n);
    out.w.resize(C.n);
    for (int c = 0; c < C.n; ++c) {
      for (int a = 0; a < 3; ++a) out.node[3 * c + a] = C.node[c][a];
      out.w[c] = C.w[c];
    }
    return true;
  }
  // tensor product of the per-axis weights, axes in (x, y, z) order
  constexpr int W = 2 * FWI_SINC_RADIUS;
  int first[3] = {0, 0, 0};
  double w1[3][W];
  for (int a = 0; a < nd; ++a) {
    const double xa = xyz[nd - 1 - a] / P->h[a];
    if (!sinc_axis(xa, P->n3[a], &first[a], w1[a])) return false;
  }
  out.n = interp_nodes(FWI_INTERP_SINC, nd);
  out.node.assign(3 * out.n, 0);
  out.w.assign(out.n, 1.0);
  for (int c = 0; c < out.n; ++c) {
    int rem = c;
    for (int a = 0; a < nd; ++a) {
      const int j = rem % W;
      rem /= W;
      out.node[3 * c + a] = first[a] + j;
      out.w[c] *= w1[a][j];
    }
  }
  return true;
}

TileGeo tile_geo(const fwi_plan* P, int tile, bool tma, bool x2, bool ext) {
  TileGeo T{};
  if (ext) {   // kernels_ext.cu: 128 x 16 tiles (2D), 32 x 8 columns in z chunks (3D)
    const bool three = P->grid.ndim == 3;
    T.tx = three ? EXT_TX : EXT_TX2;
    T.ty = three ? EXT_TY3 : EXT_TY2;
    T.zc = three ? EXT_ZC : 1;
    T.gx = (P->L.nx + T.tx - 1) / T.tx;
    T.gy = (P->L.ny + T.ty - 1) / T.ty;
    T.nzc = three ? (P->L.nz + T.zc - 1) / T.zc : 1;
    return T;
  }
  if (P->grid.ndim == 2) {
    const Tile2 t = tma ? tile2_tma_variant(tile) : tile2_variant(tile);
    T.tx = TILE_X;
    T.ty = t.ry * t.by;
    T.zc = 1;
    T.gx = (P->L.nx + T.tx - 1) / T.tx;
    T.gy = (P->L.ny + T.ty - 1) / T.ty;
    T.nzc = 1;
  } else {
    const Tile3 t = tile3_variant(tile);
    T.tx = x2 ? 64 : 32;   // the two-point kernels cover 64 x points per CTA row
    T.ty = t.by;
    T.zc = t.zc;
    T.gx = (P->L.nx + T.tx - 1) / T.tx;
    T.gy = (P->L.ny + T.ty - 1) / T.ty;
    T.nzc = (P->L.nz + T.zc - 1) / T.zc;
  }
  return T;
}

void add_entry(std::vector<Entry>& E, const TileGeo& T, int slot, const int* node, int vidx,
               float w) {
  const int x = node[0], y = node[1], z = node[2];
  const int bx = x / T.tx, by = y / T.ty, bz = z / T.zc;
  const int tile = (bz * T.gy + by) * T.gx + bx;
  const int loc = ((z - bz * T.zc) * T.ty + (y - by * T.ty)) * T.tx + (x - bx * T.tx);
  E.push_back({slot * T.ntiles() + tile, loc, vidx, w});
}

HostTable bucket(const std::vector<Entry>& E_in, int nbuckets, int rows, int tx) {
  // within a bucket, entries in increasing tile-local index (the 3D kernels
  // walk them plane by plane with one cursor); stable, so the entries of one
  // node keep their order and its sum the same rounding
  std::vector<Entry> E(E_in);
  std::stable_sort(E.begin(), E.end(), [](const Entry& a, const Entry& b) {
    return a.bucket != b.bucket ? a.bucket < b.bucket : a.loc < b.loc;
  });
  HostTable H;
  H.off.assign(nbuckets + 1, 0);
  for (const Entry& e : E) H.off[e.bucket + 1]++;
  for (int i = 0; i < nbuckets; ++i) H.off[i + 1] += H.off[i];
  std::vector<int> pos(H.off.begin(), H.off.end() - 1);
  H.loc.resize(E.size());
  H.vidx.resize(E.size());
  H.w.resize(E.size());
  for (const Entry& e : E) {  // stable: keeps insertion order within a bucket
    const int k = pos[e.bucket]++;
    H.loc[k] = e.loc;
    H.vidx[k] = e.vidx;
    H.w[k] = e.w;
  }
  if (rows > 0) {   // entries of tile row r of bucket b: [row[b (rows+1) + r], row[b (rows+1) + r + 1])
    H.row.assign((size_t)nbuckets * (rows + 1), 0);
    for (int b = 0; b < nbuckets; ++b) {
      int k = H.off[b];
      for (int r = 0; r <= rows; ++r) {
        while (k < H.off[b + 1] && H.loc[k] < r * tx) ++k;
        H.row[(size_t)b * (rows + 1) + r] = k;
        if (r > 0) H.max_row = std::max(H.max_row, k - H.row[(size_t)b * (rows + 1) + r - 1]);
      }
    }
  }
  return H;
}

size_t table_bytes(const HostTable& H) {
  return align_up(H.off.size() * 4, 256) + align_up(H.loc.size() * 4 + 4, 256) * 2 +
         align_up(H.w.size() * 4 + 4, 256) + align_up(H.row.size() * 4 + 4, 256);
}

fwi_status upload_table(fwi_plan* P, const HostTable& H, Carve& C, DevTable& D) {
  int* off = C.take<int>(H.off.size());
  int* loc = C.take<int>(H.loc.size() + 1);
  int* vidx = C.take<int>(H.vidx.size() + 1);
  float* w = C.take<float>(H.w.size() + 1);
  CUDA_TRY(cudaMemcpyAsync(off, H.off.data(), H.off.size() * 4, cudaMemcpyHostToDevice, P->st));
  if (!H.loc.empty()) {
    CUDA_TRY(cudaMemcpyAsync(loc, H.loc.data(), H.loc.size() * 4, cudaMemcpyHostToDevice, P->st));
    CUDA_TRY(cudaMemcpyAsync(vidx, H.vidx.data(), H.vidx.size() * 4, cudaMemcpyHostToDevice, P->st));
    CUDA_TRY(cudaMemcpyAsync(w, H.w.data(), H.w.size() * 4, cudaMemcpyHostToDevice, P->st));
  }
  D.off = off;
  D.loc = loc;
  D.vidx = vidx;
  D.w = w;
  D.row = nullptr;
  D.crowded = H.max_row > 32;
  if (!H.row.empty()) {
    int* row = C.take<int>(H.row.size());
    CUDA_TRY(cudaMemcpyAsync(row, H.row.data(), H.row.size() * 4, cudaMemcpyHostToDevice, P->st));
    D.row = row;
  }
  return FWI_OK;
}

fwi_status build_source_table(Call& c, int shot0, int nb, Carve& C, DevTable& D) {
  fwi_plan* P = c.P;
  const fwi_geometry* g = c.geom;
  const int nd = P->grid.ndim;
  double dV = 1.0;
  for (int a = 0; a < nd; ++a) dV *= P->h[a];
  std::vector<Entry> E;
  E.reserve((size_t)nb * g->nsrc * c.ncorner);
  PointSt ps;
  for (int b = 0; b < nb; ++b) {
    const int s = shot0 + b;
    for (int k = 0; k < g->nsrc; ++k) {
      if (!point_stencil(P, g->src_xyz + ((long long)s * g->nsrc + k) * nd, ps))
        return fail(FWI_ERR_INVALID_ARG, "a sinc source lies too close to a face");
      for (int q = 0; q < ps.n; ++q)
        add_entry(E, c.T, b, &ps.node[3 * q], (s * g->nsrc + k) * P->nt, (float)(ps.w[q] / dV));
    }
  }
  const HostTable H = bucket(E, c.pl.B * c.T.ntiles(), P->grid.ndim == 2 ? c.T.ty : 0, c.T.tx);
  return upload_table(P, H, C, D);
}

// Sampling table of the sources of shots shot0 .. shot0+nb-1: per (slot,
// source) point its corner nodes and weight / cell volume (the transpose of
// the injection, so that sampling an adjoint field there gives dJ/dq).
fwi_status build_source_sampling(Call& c, int shot0, int nb, int* d_node, float* d_w) {
  fwi_plan* P = c.P;
  const fwi_geometry* g = c.geom;
  const int nd = P->grid.ndim;
  double dV = 1.0;
  for (int a = 0; a < nd; ++a) dV *= P->h[a];
  std::vector<int> node((size_t)nb * g->nsrc * c.ncorner, 0);
  std::vector<float> w(node.size(), 0.f);
  PointSt ps;
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < g->nsrc; ++k) {
      if (!point_stencil(P, g->src_xyz + ((long long)(shot0 + b) * g->nsrc + k) * nd, ps))
        return fail(FWI_ERR_INVALID_ARG, "a sinc source lies too close to a face");
      const size_t pt = (size_t)b * g->nsrc + k;
      for (int q = 0; q < ps.n; ++q) {
        node[pt * c.ncorner + q] = (int)node_index(P->L, &ps.node[3 * q]);
        w[pt * c.ncorner + q] = (float)(ps.w[q] / dV);
      }
    }
  // pageable sources: the copies have staged them when cudaMemcpyAsync returns
  CUDA_TRY(cudaMemcpyAsync(d_node, node.data(), node.size() * 4, cudaMemcpyHostToDevice, P->st));
  CUDA_TRY(cudaMemcpyAsync(d_w, w.data(), w.size() * 4, cudaMemcpyHostToDevice, P->st));
  CUDA_TRY(cudaStreamSynchronize(P->st));
  c.ws_node = d_node;
  c.ws_w = d_w;
  return FWI_OK;
}

fwi_status prepare_common(Call& c, Carve& tabC) {
  fwi_plan* P = c.P;
  const fwi_geometry* g = c.geom;
  const int nd = P->grid.ndim;
  c.ncorner = interp_nodes(P->opt.interp, nd);
  c.T = tile_geo(P, c.pl.shape, c.pl.tma, c.pl.x2, c.pl.sc.ext() && !c.pl.tma);
  // receiver sampling table
  std::vector<int> node((size_t)g->nrec * c.ncorner);
  std::vector<float> w((size_t)g->nrec * c.ncorner);
  std::vector<Entry> E;
  PointSt ps;
  for (int r = 0; r < g->nrec; ++r) {
    if (!point_stencil(P, g->rec_xyz + (long long)r * nd, ps))
      return fail(FWI_ERR_INVALID_ARG, "a sinc receiver lies too close to a face");
    for (int q = 0; q < ps.n; ++q) {
      node[(size_t)r * c.ncorner + q] = (int)node_index(P->L, &ps.node[3 * q]);
      w[(size_t)r * c.ncorner + q] = (float)ps.w[q];
    }
    if (c.pl.gradient)
      for (int b = 0; b < c.pl.B; ++b)
        for (int q = 0; q < ps.n; ++q)
          add_entry(E, c.T, b, &ps.node[3 * q], b * g->nrec + r, (float)ps.w[q]);
  }
  if (P->L.fstride >= (1LL << 31)) return fail(FWI_ERR_UNSUPPORTED, "field larger than 2^31 points");
  int* dn = tabC.take<int>(node.size());
  float* dw = tabC.take<float>(w.size());
  CUDA_TRY(cudaMemcpyAsync(dn, node.data(), node.size() * 4, cudaMemcpyHostToDevice, P->st));
  CUDA_TRY(cudaMemcpyAsync(dw, w.data(), w.size() * 4, cudaMemcpyHostToDevice, P->st));
  c.smp_node = dn;
  c.smp_w = dw;
  if (c.pl.gradient) {
    const HostTable H = bucket(E, c.pl.B * c.T.ntiles(), nd == 2 ? c.T.ty : 0, c.T.tx);
    FWI_TRY(upload_table(P, H, tabC, c.rec_tab));
  }
  return FWI_OK;
}

size_t tables_bound(const fwi_plan* P, const fwi_geometry* g, const Plan& pl) {
  const TileGeo T = tile_geo(P, pl.shape, pl.tma, pl.x2, pl.sc.ext() && !pl.tma);
  const int nc = interp_nodes(P->opt.interp, P->grid.ndim);
  const size_t nb = (size_t)pl.B * T.ntiles() + 1;
  const size_t src = (size_t)pl.B * g->nsrc * nc;
  const size_t rec = (size_t)g->nrec * nc;
  const size_t rows = P->grid.ndim == 2 ? nb * (T.ty + 1) * 4 * 2 + 2 * 256 : 0;   // per-row ranges
  return 8 * 256 + nb * 4 * 2 + (src + 1) * 12 + rec * 8 + (pl.gradient ? rec * pl.B * 12 + 4096 : 0) +
         4096 * 4 + rows;
}

}  // namespace fwi

using namespace fwi;

extern "C" {

fwi_status fwi_point_weights(const fwi_grid* grid, const double* xyz, int interp,
                             int64_t* nodes, double* weights, int cap, int* count) {
  if (count) *count = 0;
  FWI_TRY(validate_grid(grid));
  if (!xyz || !count) return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: NULL argument");
  if (interp != FWI_INTERP_LINEAR && interp != FWI_INTERP_SINC)
    return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: interp must be FWI_INTERP_LINEAR or FWI_INTERP_SINC");
  const int nd = grid->ndim;
  for (int d = 0; d < nd; ++d) {
    const double hi = (double)(grid->shape[d] - 1) * grid->spacing[d];
    const double tol = 1e-9 * grid->spacing[d];
    if (!std::isfinite(xyz[d]) || xyz[d] < -tol || xyz[d] > hi + tol)
      return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: point outside the grid");
  }
  if (interp == FWI_INTERP_LINEAR) {
    fwi_plan P;   // only the layout fields are used (no device work)
    P.grid = *grid;
    build_layout(&P);
    const Corners C = point_corners(&P, xyz);
    *count = C.n;
    if (cap < C.n || !nodes || !weights)
      return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: cap below count (count is set)");
    for (int c = 0; c < C.n; ++c) {
      for (int d = 0; d < nd; ++d) nodes[(size_t)c * nd + d] = C.node[c][nd - 1 - d];
      weights[c] = C.w[c];
    }
    return FWI_OK;
  }
  // Kaiser-windowed sinc: per axis the 2r nodes floor(x)-r+1 .. floor(x)+r;
  // the point weights are the products over the axes.
  constexpr int r = FWI_SINC_RADIUS;
  int first[3] = {0, 0, 0};
  double w1[3][2 * FWI_SINC_RADIUS];
  int total = 1;
  for (int d = 0; d < nd; ++d) {
    if (!sinc_axis(xyz[d] / grid->spacing[d], grid->shape[d], &first[d], w1[d]))
      return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: a sinc point must lie r - 1 nodes inside every face");
    total *= 2 * r;
  }
  *count = total;
  if (cap < total || !nodes || !weights)
    return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: cap below count (count is set)");
  for (int c = 0; c < total; ++c) {         // the slowest axis varies slowest
    int rem = c;
    double w = 1.0;
    for (int d = nd - 1; d >= 0; --d) {
      const int j = rem % (2 * r);
      rem /= 2 * r;
      nodes[(size_t)c * nd + d] = first[d] + j;
      w *= w1[d][j];
    }
    weights[c] = w;
  }
  return FWI_OK;
}

}  // extern "C"
