// C ABI of the GB300 acoustic FWI library: plans, validation, workspace,
// shot batching and the forward / gradient drivers (see include/fwi.h).
//
// Forward modelling and the adjoint-state gradient follow Sec. 2.2 (Eqs.
// 5-9) and Sec. 2.4 (Eq. 10) of the Stride paper: per shot, one forward
// propagation storing h^n = k (L u^n + s^n) (or checkpoints of (u^n, u^{n-1})
// every K steps with per-segment recomputation), the L2 residual, and one
// adjoint propagation backwards in time with the imaging condition fused
// into the adjoint step.  Shots run as a batch dimension of every launch.
#include "fwi.h"
#include "fwi_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace fwi;

namespace {

thread_local std::string g_err;

fwi_status fail(fwi_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(FWI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define FWI_TRY(call)                \
  do {                               \
    fwi_status s_ = (call);          \
    if (s_ != FWI_OK) return s_;     \
  } while (0)

// Central-difference weights (standard Taylor weights of the stated order):
// second derivative w2[0..R], first derivative w1[1..R] (antisymmetric).
void fd_weights(int order, double* w2, double* w1) {
  for (int j = 0; j < 6; ++j) w2[j] = w1[j] = 0.0;
  if (order == 8) {
    const double a[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    const double b[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
    for (int j = 0; j < 5; ++j) { w2[j] = a[j]; w1[j] = b[j]; }
  } else {
    const double a[6] = {-5269.0 / 1800.0, 5.0 / 3.0, -5.0 / 21.0, 5.0 / 126.0, -5.0 / 1008.0,
                         1.0 / 3150.0};
    const double b[6] = {0.0, 5.0 / 6.0, -5.0 / 21.0, 5.0 / 84.0, -5.0 / 504.0, 1.0 / 1260.0};
    for (int j = 0; j < 6; ++j) { w2[j] = a[j]; w1[j] = b[j]; }
  }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round_up(int v, int a) { return (v + a - 1) / a * a; }

}  // namespace

struct fwi_plan {
  fwi_grid grid{};
  int nt = 0;
  double dt = 0.0;
  size_t budget = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  fwi_options opt{};
  fwi_stats stats{};
  Layout L{};
  int R = 4;
  double h[3] = {1, 1, 1};  // spacing (x, y, z)
  int n3[3] = {1, 1, 1};    // extents (x, y, z)
  double c_ref = 0.0;
  bool sponge_ready = false;
  AxisW wx{}, wy{}, wz{};
  float* spx = nullptr;
  float* spy = nullptr;
  float* spz = nullptr;
  unsigned int* d_stats = nullptr;
  int* d_flags = nullptr;
  double* d_J = nullptr;     // per-batch misfit
  int d_J_cap = 0;
  char* arena = nullptr;
  size_t arena_cap = 0;
  // small device tables (grown on demand)
  char* tab = nullptr;
  size_t tab_cap = 0;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;  // 0 forward, 1 adjoint
  size_t ev_used = 0;
};

namespace {

struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

fwi_status ensure_arena(fwi_plan* P, size_t bytes) {
  if (bytes <= P->arena_cap) return FWI_OK;
  if (P->arena) {
    CUDA_TRY(cudaStreamSynchronize(P->st));
    CUDA_TRY(cudaFree(P->arena));
    P->arena = nullptr;
    P->arena_cap = 0;
  }
  cudaError_t e = cudaMalloc(&P->arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    P->arena = nullptr;
    return fail(FWI_ERR_BUDGET, "workspace allocation of " + std::to_string(bytes) +
                                    " bytes failed: " + cudaGetErrorString(e));
  }
  P->arena_cap = bytes;
  return FWI_OK;
}

fwi_status ensure_tab(fwi_plan* P, size_t bytes) {
  if (bytes <= P->tab_cap) return FWI_OK;
  if (P->tab) {
    CUDA_TRY(cudaStreamSynchronize(P->st));
    CUDA_TRY(cudaFree(P->tab));
    P->tab = nullptr;
  }
  bytes = std::max(bytes, (size_t)1 << 20);
  CUDA_TRY(cudaMalloc(&P->tab, bytes));
  P->tab_cap = bytes;
  return FWI_OK;
}

// Bi-/tri-linear stencil of one point: nodes (x, y, z) and weights.
struct Corners {
  int n;
  int node[8][3];
  double w[8];
};

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

// Tile geometry of the stencil kernels for entry bucketing.
struct TileGeo {
  int gx, gy, nzc, tx, ty, zc;
  int ntiles() const { return gx * gy * nzc; }
};

TileGeo tile_geo(const fwi_plan* P, int tile) {
  TileGeo T{};
  if (P->grid.ndim == 2) {
    const Tile2 t = tile2_variant(tile);
    T.tx = TILE_X;
    T.ty = t.ry * t.by;
    T.zc = 1;
    T.gx = (P->L.nx + T.tx - 1) / T.tx;
    T.gy = (P->L.ny + T.ty - 1) / T.ty;
    T.nzc = 1;
  } else {
    const Tile3 t = tile3_variant(tile);
    T.tx = 32;
    T.ty = t.by;
    T.zc = t.zc;
    T.gx = (P->L.nx + 31) / 32;
    T.gy = (P->L.ny + T.ty - 1) / T.ty;
    T.nzc = (P->L.nz + T.zc - 1) / T.zc;
  }
  return T;
}

struct Entry {
  int bucket;
  int loc;
  int vidx;
  float w;
};

void add_entry(std::vector<Entry>& E, const TileGeo& T, int slot, const int* node, int vidx,
               float w) {
  const int x = node[0], y = node[1], z = node[2];
  const int bx = x / T.tx, by = y / T.ty, bz = z / T.zc;
  const int tile = (bz * T.gy + by) * T.gx + bx;
  const int loc = ((z - bz * T.zc) * T.ty + (y - by * T.ty)) * T.tx + (x - bx * T.tx);
  E.push_back({slot * T.ntiles() + tile, loc, vidx, w});
}

// Host-side bucket tables, laid out [off | loc | vidx | w].
struct HostTable {
  std::vector<int> off, loc, vidx;
  std::vector<float> w;
};

HostTable bucket(const std::vector<Entry>& E, int nbuckets) {
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
  return H;
}

struct DevTable {
  const int* off = nullptr;
  const int* loc = nullptr;
  const int* vidx = nullptr;
  const float* w = nullptr;
};

size_t table_bytes(const HostTable& H) {
  return align_up(H.off.size() * 4, 256) + align_up(H.loc.size() * 4 + 4, 256) * 2 +
         align_up(H.w.size() * 4 + 4, 256);
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
  return FWI_OK;
}

double cfl_limit(int ndim, int order) {
  double w2[6], w1[6];
  fd_weights(order, w2, w1);
  const int R = order / 2;
  double lam = w2[0];
  for (int j = 1; j <= R; ++j) lam += 2.0 * ((j & 1) ? -w2[j] : w2[j]);
  lam = std::fabs(lam);
  return 2.0 / std::sqrt(ndim * lam);
}

fwi_status validate_grid(const fwi_grid* g) {
  if (!g) return fail(FWI_ERR_INVALID_ARG, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(FWI_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (g->order != 8 && g->order != 10) return fail(FWI_ERR_INVALID_ARG, "order must be 8 or 10");
  for (int d = 0; d < g->ndim; ++d) {
    if (g->shape[d] < 4 || g->shape[d] > (1 << 20))
      return fail(FWI_ERR_INVALID_ARG, "shape out of range [4, 2^20]");
    if (!(g->spacing[d] > 0.0) || !std::isfinite(g->spacing[d]))
      return fail(FWI_ERR_INVALID_ARG, "spacing must be positive and finite");
    if (g->sponge < 0 || 2 * (int64_t)g->sponge >= g->shape[d])
      return fail(FWI_ERR_INVALID_ARG, "sponge must be >= 0 and < shape/2");
  }
  long long N = 1;
  for (int d = 0; d < g->ndim; ++d) N *= g->shape[d];
  if (N > (1LL << 34)) return fail(FWI_ERR_INVALID_ARG, "grid too large");
  return FWI_OK;
}

void build_layout(fwi_plan* P) {
  const fwi_grid& g = P->grid;
  Layout& L = P->L;
  L.ndim = g.ndim;
  P->R = g.order / 2;
  L.R = P->R;
  if (g.ndim == 2) {
    L.ny = (int)g.shape[0];
    L.nx = (int)g.shape[1];
    L.nz = 1;
    P->h[1] = g.spacing[0];
    P->h[0] = g.spacing[1];
    P->h[2] = 1.0;
  } else {
    L.nz = (int)g.shape[0];
    L.ny = (int)g.shape[1];
    L.nx = (int)g.shape[2];
    P->h[2] = g.spacing[0];
    P->h[1] = g.spacing[1];
    P->h[0] = g.spacing[2];
  }
  P->n3[0] = L.nx;
  P->n3[1] = L.ny;
  P->n3[2] = L.nz;
  L.nx_r = round_up(L.nx, TILE_X);
  L.ny_r = round_up(L.ny, ROUND_Y);
  L.nz_r = L.nz;
  L.ox = OX;
  L.sx = OX + L.nx_r + 8;
  L.oy = P->R;
  L.rows = L.oy + L.ny_r + P->R;
  L.oz = (g.ndim == 3) ? P->R : 0;
  L.planes = (g.ndim == 3) ? L.oz + L.nz + P->R : 1;
  L.sxy = (long long)L.sx * L.rows;
  L.fstride = (long long)align_up((size_t)(L.sxy * L.planes), 64);
  double w2[6], w1[6];
  fd_weights(g.order, w2, w1);
  AxisW* W[3] = {&P->wx, &P->wy, &P->wz};
  for (int a = 0; a < 3; ++a) {
    for (int j = 0; j < 6; ++j) {
      const bool on = a < g.ndim && j <= P->R;
      W[a]->w2[j] = on ? (float)(w2[j] / (P->h[a] * P->h[a])) : 0.f;
      W[a]->w1[j] = on ? (float)(w1[j] / P->h[a]) : 0.f;
    }
  }
}

// a_d(i) = sigma_d(i) dt / 2 with sigma_d = smax_d (delta/nb)^2,
// smax_d = 3 c_ref ln(1000) / (2 nb h_d); delta = points into the layer.
fwi_status build_sponge(fwi_plan* P) {
  const int nb = P->grid.sponge;
  const int len[3] = {P->L.nx_r, P->L.ny_r, std::max(P->L.nz, 1)};
  float** dst[3] = {&P->spx, &P->spy, &P->spz};
  for (int a = 0; a < 3; ++a) {
    std::vector<float> v(len[a] + 8, 0.f);
    const int n = P->n3[a];
    if (a < P->grid.ndim && nb > 0) {
      const double smax = 3.0 * P->c_ref * std::log(1000.0) / (2.0 * nb * P->h[a]);
      for (int i = 0; i < n; ++i) {
        int delta = 0;
        if (i < nb) delta = nb - i;
        else if (i > n - 1 - nb) delta = i - (n - 1 - nb);
        const double r = (double)delta / nb;
        v[i] = (float)(smax * r * r * P->dt * 0.5);
      }
    }
    if (!*dst[a]) CUDA_TRY(cudaMalloc(dst[a], v.size() * sizeof(float)));
    CUDA_TRY(cudaMemcpy(*dst[a], v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  P->sponge_ready = true;
  return FWI_OK;
}

fwi_status validate_geometry(const fwi_plan* P, const fwi_geometry* g) {
  if (!g) return fail(FWI_ERR_INVALID_ARG, "geometry is NULL");
  if (g->nshots < 1 || g->nsrc < 1 || g->nrec < 1)
    return fail(FWI_ERR_INVALID_ARG, "nshots, nsrc and nrec must be >= 1");
  if (!g->src_xyz || !g->rec_xyz) return fail(FWI_ERR_INVALID_ARG, "coordinates are NULL");
  if ((long long)g->nshots * g->nsrc > (1LL << 24) || g->nrec > (1 << 24))
    return fail(FWI_ERR_INVALID_ARG, "too many sources or receivers");
  const int nd = P->grid.ndim;
  auto check = [&](const double* p) {
    for (int d = 0; d < nd; ++d) {
      const double hi = (double)(P->grid.shape[d] - 1) * P->grid.spacing[d];
      const double tol = 1e-9 * P->grid.spacing[d];
      if (!std::isfinite(p[d]) || p[d] < -tol || p[d] > hi + tol) return false;
    }
    return true;
  };
  for (long long i = 0; i < (long long)g->nshots * g->nsrc; ++i)
    if (!check(g->src_xyz + i * nd))
      return fail(FWI_ERR_INVALID_ARG, "source " + std::to_string(i) + " lies outside the grid");
  for (int i = 0; i < g->nrec; ++i)
    if (!check(g->rec_xyz + (long long)i * nd))
      return fail(FWI_ERR_INVALID_ARG, "receiver " + std::to_string(i) + " lies outside the grid");
  return FWI_OK;
}

// Workspace plan for one call.
struct Plan {
  int B = 1;            // slots
  int K = 0;            // 0: full history; else checkpoint interval
  int nck = 0;          // checkpoints per shot
  bool gradient = false;
  int tile = 0;
  size_t bytes = 0;
};

size_t field_bytes(const fwi_plan* P) { return (size_t)P->L.fstride * sizeof(float); }

size_t model_bytes(const fwi_plan* P, bool vd) {
  const size_t f = align_up(field_bytes(P), 256);
  return f * (1 + (vd ? 1 + P->grid.ndim : 0));
}

size_t slot_bytes(const fwi_plan* P, const fwi_geometry* g, bool grad, int K) {
  const size_t f = align_up(field_bytes(P), 256);
  const size_t traces = align_up((size_t)P->nt * g->nrec * sizeof(float), 256);
  size_t b = 2 * f + traces;
  if (!grad) return b;
  b += f;  // g slot
  const int nt = P->nt;
  if (K == 0) {
    b += (size_t)std::max(nt - 1, 1) * f;
  } else {
    const int nck = (nt - 2) / K + 1;
    b += 2 * f + 2 * (size_t)nck * f + (size_t)K * f;
  }
  return b;
}

size_t fixed_bytes(const fwi_plan* P, const fwi_geometry* g, bool vd, int B) {
  const size_t misfit = align_up((size_t)misfit_blocks(B, g->nrec, P->nt) * 8, 256);
  return model_bytes(P, vd) + misfit + (4u << 20);
}

fwi_status choose_plan(const fwi_plan* P, const fwi_geometry* g, bool vd, bool grad, Plan& out) {
  const int ns = g->nshots;
  const size_t budget = P->budget;
  const int K_auto = std::max(2, (int)std::ceil(std::sqrt(2.0 * std::max(P->nt, 2))));
  const long long N = (long long)P->L.nx * P->L.ny * P->L.nz;
  const int B_fill = (int)std::max(1LL, (8LL << 20) / std::max(N, 1LL));  // slots that fill the GPU
  auto fit = [&](int K) {
    const size_t fixed = fixed_bytes(P, g, vd, ns);
    if (budget <= fixed) return 0;
    const size_t per = slot_bytes(P, g, grad, K);
    return (int)std::min<size_t>((size_t)ns, (budget - fixed) / per);
  };
  int K = 0;
  if (grad) {
    if (P->opt.ckpt_every > 0) K = std::min(P->opt.ckpt_every, std::max(P->nt - 1, 1));
    else if (P->opt.ckpt_every < 0) K = 0;
    else {
      const int want = std::min(ns, P->opt.batch > 0 ? P->opt.batch : B_fill);
      K = (fit(0) >= want) ? 0 : K_auto;
    }
    if (K >= P->nt - 1) K = 0;
  }
  int B = fit(K);
  if (B < 1) return fail(FWI_ERR_BUDGET, "one shot does not fit the HBM budget (" +
                                             std::to_string(budget) + " bytes)");
  if (P->opt.batch > 0) B = std::min(B, P->opt.batch);
  B = std::min(B, ns);
  out.B = B;
  out.K = K;
  out.nck = K ? (P->nt - 2) / K + 1 : 0;
  out.gradient = grad;
  out.tile = P->opt.tile;
  out.bytes = fixed_bytes(P, g, vd, B) + (size_t)B * slot_bytes(P, g, grad, K);
  return FWI_OK;
}

// Per-call device state carved out of the arena.
struct Work {
  float *kf = nullptr, *lnr = nullptr, *bx = nullptr, *by = nullptr, *bz = nullptr;
  float *U0 = nullptr, *U1 = nullptr, *F0 = nullptr, *F1 = nullptr, *G = nullptr;
  float *H = nullptr, *CK = nullptr, *D = nullptr;
  double* partials = nullptr;
  int npartials = 0;
};

void carve_work(fwi_plan* P, const Plan& pl, const fwi_geometry* g, bool vd, Carve& C, Work& W) {
  const size_t fs = (size_t)P->L.fstride;
  const int B = pl.B;
  W.kf = C.take<float>(fs);
  if (vd) {
    W.lnr = C.take<float>(fs);
    W.bx = C.take<float>(fs);
    W.by = C.take<float>(fs);
    if (P->grid.ndim == 3) W.bz = C.take<float>(fs);
  }
  W.npartials = misfit_blocks(B, g->nrec, P->nt);
  W.partials = C.take<double>(W.npartials);
  W.U0 = C.take<float>(fs * B);
  W.U1 = C.take<float>(fs * B);
  W.D = C.take<float>((size_t)P->nt * B * g->nrec);
  if (pl.gradient) {
    W.G = C.take<float>(fs * B);
    if (pl.K == 0) {
      W.H = C.take<float>(fs * B * (size_t)std::max(P->nt - 1, 1));
    } else {
      W.F0 = C.take<float>(fs * B);
      W.F1 = C.take<float>(fs * B);
      W.CK = C.take<float>(fs * B * 2 * (size_t)pl.nck);
      W.H = C.take<float>(fs * B * (size_t)pl.K);
    }
  }
}

struct Call {
  fwi_plan* P;
  const fwi_model* model;
  const fwi_geometry* geom;
  const float* wavelet;
  bool vd;
  Plan pl;
  Work W;
  TileGeo T;
  DevTable smp_tab;   // receiver sampling: node/w only (off unused)
  const int* smp_node = nullptr;
  const float* smp_w = nullptr;
  DevTable rec_tab;   // adjoint residual injection, per slot
  int ncorner = 4;
  int64_t launches = 0;
  int64_t fwd_launches = 0, adj_launches = 0;
  int64_t fwd_points = 0, adj_points = 0;
};

fwi_status record_event(fwi_plan* P, int kind) {
  if (P->ev_used >= P->ev.size()) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    P->ev.push_back(e);
    P->ev_kind.push_back(kind);
  }
  P->ev_kind[P->ev_used] = kind;
  CUDA_TRY(cudaEventRecord(P->ev[P->ev_used], P->st));
  P->ev_used++;
  return FWI_OK;
}

StepParams base_params(Call& c) {
  fwi_plan* P = c.P;
  StepParams p{};
  p.kf = c.W.kf;
  p.bx = c.W.bx;
  p.by = c.W.by;
  p.bz = c.W.bz;
  p.spx = P->spx;
  p.spy = P->spy;
  p.spz = P->spz;
  p.fstride = P->L.fstride;
  p.sxy = P->L.sxy;
  p.sx = P->L.sx;
  p.nx = P->L.nx;
  p.ny = P->L.ny;
  p.nz = P->L.nz;
  p.ox = P->L.ox;
  p.oy = P->L.oy;
  p.oz = P->L.oz;
  p.wx = P->wx;
  p.wy = P->wy;
  p.wz = P->wz;
  p.ntiles = c.T.ntiles();
  p.ncorner = c.ncorner;
  if (P->grid.ndim == 3) {
    p.zchunk = c.T.zc;
    p.nzc = c.T.nzc;
  } else {
    p.zchunk = 1;
    p.nzc = 1;
  }
  return p;
}

long long launch_threads(const Call& c, int B) {
  const int by = (c.P->grid.ndim == 2) ? tile2_variant(c.pl.tile).by : tile3_variant(c.pl.tile).by;
  return (long long)c.T.ntiles() * B * 32 * by;
}

fwi_status launch_step(Call& c, const StepParams& p_in, bool adj) {
  fwi_plan* P = c.P;
  StepParams p = p_in;
  if (!adj && p.nrec > 0 && (long long)p.B * p.nrec > launch_threads(c, p.B)) {
    // too few threads in the stencil launch to sample every receiver: do it apart
    cudaError_t e = launch_sample(p, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
    p.nrec = 0;
  }
  const bool prof = P->opt.profile != 0;
  if (prof) FWI_TRY(record_event(P, adj ? 1 : 0));
  cudaError_t e = (P->grid.ndim == 2) ? launch_step2d(p, P->R, c.vd, adj, c.pl.tile, P->st)
                                      : launch_step3d(p, P->R, c.vd, adj, c.pl.tile, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("stencil launch: ") + cudaGetErrorString(e));
  if (prof) FWI_TRY(record_event(P, adj ? 1 : 0));
  c.launches++;
  const int64_t pts = (int64_t)p.B * P->L.nx * P->L.ny * P->L.nz;
  if (adj) { c.adj_launches++; c.adj_points += pts; }
  else { c.fwd_launches++; c.fwd_points += pts; }
  return FWI_OK;
}

// Forward sweep of one batch: steps n = n0 .. n1-1 starting from (A = u^{n0},
// Bf = u^{n0-1}).  hist_base: full history [n][B][fs] (n indexed from 0) or a
// segment buffer indexed from n0; sample: record d^n for each step.
fwi_status forward_steps(Call& c, int nb, int shot0, const DevTable& src, float*& A, float*& Bf,
                         int n0, int n1, float* hist_base, int hist_n0, bool sample,
                         int K_ckpt, float* CK) {
  fwi_plan* P = c.P;
  const size_t fs = (size_t)P->L.fstride;
  StepParams p = base_params(c);
  p.B = nb;
  p.inj_off = src.off;
  p.inj_loc = src.loc;
  p.inj_vidx = src.vidx;
  p.inj_w = src.w;
  p.vals = c.wavelet;
  p.smp_node = c.smp_node;
  p.smp_w = c.smp_w;
  p.smp_out = c.W.D;
  p.nrec = sample ? c.geom->nrec : 0;
  for (int n = n0; n < n1; ++n) {
    if (K_ckpt > 0 && n % K_ckpt == 0) {
      const size_t j = n / K_ckpt;
      float* dst = CK + 2 * j * fs * c.pl.B;
      CUDA_TRY(cudaMemcpyAsync(dst, A, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
      CUDA_TRY(cudaMemcpyAsync(dst + fs * c.pl.B, Bf, fs * nb * sizeof(float),
                               cudaMemcpyDeviceToDevice, P->st));
    }
    p.u = A;
    p.up = Bf;
    p.hist = hist_base ? hist_base + (size_t)(n - hist_n0) * fs * c.pl.B : nullptr;
    p.step_off = n;
    p.smp_off = (long long)n * c.pl.B * c.geom->nrec;
    FWI_TRY(launch_step(c, p, false));
    std::swap(A, Bf);
  }
  (void)shot0;
  return FWI_OK;
}

fwi_status final_sample(Call& c, int nb, const float* A, int n) {
  fwi_plan* P = c.P;
  StepParams p = base_params(c);
  p.B = nb;
  p.u = A;
  p.smp_node = c.smp_node;
  p.smp_w = c.smp_w;
  p.smp_out = c.W.D;
  p.nrec = c.geom->nrec;
  p.smp_off = (long long)n * c.pl.B * c.geom->nrec;
  cudaError_t e = launch_sample(p, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  c.launches++;
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
  for (int b = 0; b < nb; ++b) {
    const int s = shot0 + b;
    for (int k = 0; k < g->nsrc; ++k) {
      const Corners cr = point_corners(P, g->src_xyz + ((long long)s * g->nsrc + k) * nd);
      for (int q = 0; q < cr.n; ++q)
        add_entry(E, c.T, b, cr.node[q], (s * g->nsrc + k) * P->nt, (float)(cr.w[q] / dV));
    }
  }
  const HostTable H = bucket(E, c.pl.B * c.T.ntiles());
  return upload_table(P, H, C, D);
}

fwi_status prepare_common(Call& c, Carve& tabC) {
  fwi_plan* P = c.P;
  const fwi_geometry* g = c.geom;
  const int nd = P->grid.ndim;
  c.ncorner = 1 << nd;
  c.T = tile_geo(P, c.pl.tile);
  // receiver sampling table
  std::vector<int> node((size_t)g->nrec * c.ncorner);
  std::vector<float> w((size_t)g->nrec * c.ncorner);
  std::vector<Entry> E;
  for (int r = 0; r < g->nrec; ++r) {
    const Corners cr = point_corners(P, g->rec_xyz + (long long)r * nd);
    for (int q = 0; q < cr.n; ++q) {
      node[(size_t)r * c.ncorner + q] = (int)node_index(P->L, cr.node[q]);
      w[(size_t)r * c.ncorner + q] = (float)cr.w[q];
    }
    if (c.pl.gradient)
      for (int b = 0; b < c.pl.B; ++b)
        for (int q = 0; q < cr.n; ++q)
          add_entry(E, c.T, b, cr.node[q], b * g->nrec + r, (float)cr.w[q]);
  }
  if (P->L.fstride >= (1LL << 31)) return fail(FWI_ERR_UNSUPPORTED, "field larger than 2^31 points");
  int* dn = tabC.take<int>(node.size());
  float* dw = tabC.take<float>(w.size());
  CUDA_TRY(cudaMemcpyAsync(dn, node.data(), node.size() * 4, cudaMemcpyHostToDevice, P->st));
  CUDA_TRY(cudaMemcpyAsync(dw, w.data(), w.size() * 4, cudaMemcpyHostToDevice, P->st));
  c.smp_node = dn;
  c.smp_w = dw;
  if (c.pl.gradient) {
    const HostTable H = bucket(E, c.pl.B * c.T.ntiles());
    FWI_TRY(upload_table(P, H, tabC, c.rec_tab));
  }
  return FWI_OK;
}

size_t tables_bound(const fwi_plan* P, const fwi_geometry* g, const Plan& pl) {
  const TileGeo T = tile_geo(P, pl.tile);
  const int nc = 1 << P->grid.ndim;
  const size_t nb = (size_t)pl.B * T.ntiles() + 1;
  const size_t src = (size_t)pl.B * g->nsrc * nc;
  const size_t rec = (size_t)g->nrec * nc;
  return 8 * 256 + nb * 4 * 2 + (src + 1) * 12 + rec * 8 + (pl.gradient ? rec * pl.B * 12 + 4096 : 0) +
         4096 * 4;
}

// Validate the model, fill k (and the density gradient), check CFL.
fwi_status prepare_model(Call& c) {
  fwi_plan* P = c.P;
  const fwi_model* m = c.model;
  const size_t fs = (size_t)P->L.fstride;
  CUDA_TRY(cudaMemsetAsync(c.W.kf, 0, fs * sizeof(float), P->st));
  unsigned int init[3] = {0u, 0x7f800000u, 0u};
  CUDA_TRY(cudaMemcpyAsync(P->d_stats, init, sizeof(init), cudaMemcpyHostToDevice, P->st));
  if (c.vd) CUDA_TRY(cudaMemsetAsync(c.W.lnr, 0, fs * sizeof(float), P->st));
  cudaError_t e = launch_model_prep(P->L, m->vp, m->rho, P->dt, c.W.kf, c.vd ? c.W.lnr : nullptr,
                                    P->d_stats, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  unsigned int st[3];
  CUDA_TRY(cudaMemcpyAsync(st, P->d_stats, sizeof(st), cudaMemcpyDeviceToHost, P->st));
  CUDA_TRY(cudaStreamSynchronize(P->st));
  if (st[2] != 0) return fail(FWI_ERR_NONFINITE, "model holds non-positive or non-finite values");
  float vmax;
  std::memcpy(&vmax, &st[0], 4);
  double sum = 0.0;
  for (int a = 0; a < P->grid.ndim; ++a) sum += 1.0 / (P->h[a] * P->h[a]);
  // stability of the leapfrog: c dt sqrt(sum 1/h^2) <= 2 / sqrt(lambda_max)
  const double lim1 = cfl_limit(1, P->grid.order);
  const double cfl = (double)vmax * P->dt * std::sqrt(sum);
  if (cfl > 0.95 * lim1) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "CFL %.4f exceeds 0.95 x leapfrog limit (%.4f) for vp_max %.1f",
                  cfl / std::sqrt((double)P->grid.ndim), 0.95 * cfl_limit(P->grid.ndim, P->grid.order),
                  (double)vmax);
    return fail(FWI_ERR_UNSTABLE_CFL, buf);
  }
  if (!P->sponge_ready) {
    if (P->c_ref <= 0.0) P->c_ref = vmax;
    FWI_TRY(build_sponge(P));
  }
  if (c.vd) {
    CUDA_TRY(cudaMemsetAsync(c.W.bx, 0, fs * sizeof(float), P->st));
    CUDA_TRY(cudaMemsetAsync(c.W.by, 0, fs * sizeof(float), P->st));
    if (c.W.bz) CUDA_TRY(cudaMemsetAsync(c.W.bz, 0, fs * sizeof(float), P->st));
    e = launch_density_grad(P->L, c.W.lnr, P->wx, P->wy, P->wz, c.W.bx, c.W.by, c.W.bz, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  }
  return FWI_OK;
}

fwi_status begin_call(fwi_plan* P, const fwi_model* model, const fwi_geometry* geom,
                      const float* wavelet, bool grad, Call& c, Carve& tabC) {
  if (!model || !model->vp) return fail(FWI_ERR_INVALID_ARG, "model or vp is NULL");
  if (!wavelet) return fail(FWI_ERR_INVALID_ARG, "wavelet is NULL");
  FWI_TRY(validate_geometry(P, geom));
  CUDA_TRY(cudaSetDevice(P->device));
  c.P = P;
  c.model = model;
  c.geom = geom;
  c.wavelet = wavelet;
  c.vd = model->rho != nullptr;
  const int ntile = P->grid.ndim == 2 ? NUM_TILE2 : NUM_TILE3;
  if (P->opt.tile < 0 || P->opt.tile >= ntile) return fail(FWI_ERR_INVALID_ARG, "tile variant out of range");
  FWI_TRY(choose_plan(P, geom, c.vd, grad, c.pl));
  FWI_TRY(ensure_arena(P, c.pl.bytes));
  Carve C(P->arena);
  carve_work(P, c.pl, geom, c.vd, C, c.W);
  if (C.off > P->arena_cap) return fail(FWI_ERR_BUDGET, "workspace carve exceeds allocation");
  FWI_TRY(ensure_tab(P, tables_bound(P, geom, c.pl) * 2));
  tabC = Carve(P->tab);
  const int nbatches = (geom->nshots + c.pl.B - 1) / c.pl.B;
  if (nbatches > P->d_J_cap) {
    if (P->d_J) CUDA_TRY(cudaFree(P->d_J));
    CUDA_TRY(cudaMalloc(&P->d_J, sizeof(double) * nbatches));
    P->d_J_cap = nbatches;
  }
  CUDA_TRY(cudaMemsetAsync(P->d_flags, 0, sizeof(int) * 4, P->st));
  P->ev_used = 0;
  FWI_TRY(prepare_model(c));
  FWI_TRY(prepare_common(c, tabC));
  return FWI_OK;
}

fwi_status finish_call(Call& c) {
  fwi_plan* P = c.P;
  int flags[4];
  CUDA_TRY(cudaMemcpyAsync(flags, P->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, P->st));
  CUDA_TRY(cudaStreamSynchronize(P->st));
  fwi_stats& s = P->stats;
  s.batch = c.pl.B;
  s.ckpt_every = c.pl.K;
  s.tile = c.pl.tile;
  s.workspace_bytes = P->arena_cap + P->tab_cap;
  s.launches = c.launches;
  s.fwd_launches = c.fwd_launches;
  s.adj_launches = c.adj_launches;
  s.fwd_points = c.fwd_points;
  s.adj_points = c.adj_points;
  s.updates = c.fwd_points + c.adj_points;
  s.fwd_ms = s.adj_ms = 0.0;
  for (size_t i = 0; i + 1 < P->ev_used; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]));
    if (P->ev_kind[i] == 0) s.fwd_ms += ms;
    else s.adj_ms += ms;
  }
  if (flags[0]) return fail(FWI_ERR_NONFINITE, "non-finite values in the result (unstable run?)");
  return FWI_OK;
}

}  // namespace

extern "C" {

const char* fwi_last_error(void) { return g_err.c_str(); }

double fwi_cfl_limit(int ndim, int order) {
  if ((ndim != 2 && ndim != 3) || (order != 8 && order != 10)) return -1.0;
  return cfl_limit(ndim, order);
}

fwi_status fwi_plan_create(fwi_plan** plan, const fwi_grid* grid, int nt, double dt,
                           size_t hbm_budget_bytes, void* stream) {
  if (!plan) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  FWI_TRY(validate_grid(grid));
  if (nt < 1 || nt > (1 << 24)) return fail(FWI_ERR_INVALID_ARG, "nt must be in [1, 2^24]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FWI_ERR_INVALID_ARG, "dt must be positive");
  fwi_plan* P = new fwi_plan();
  P->grid = *grid;
  P->nt = nt;
  P->dt = dt;
  P->st = reinterpret_cast<cudaStream_t>(stream);
  P->c_ref = grid->c_ref;
  build_layout(P);
  auto cleanup = [&](fwi_status s) { fwi_plan_destroy(P); return s; };
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) return cleanup(fail(FWI_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)));
  size_t fr = 0, tot = 0;
  e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) return cleanup(fail(FWI_ERR_CUDA, cudaGetErrorString(e)));
  P->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  if (cudaMalloc(&P->d_stats, 64) != cudaSuccess || cudaMalloc(&P->d_flags, 64) != cudaSuccess)
    return cleanup(fail(FWI_ERR_CUDA, "small allocation failed"));
  if (P->c_ref > 0.0) {
    fwi_status s = build_sponge(P);
    if (s != FWI_OK) return cleanup(s);
  }
  *plan = P;
  return FWI_OK;
}

fwi_status fwi_plan_set_options(fwi_plan* plan, const fwi_options* opt) {
  if (!plan || !opt) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  if (opt->batch < 0) return fail(FWI_ERR_INVALID_ARG, "batch must be >= 0");
  plan->opt = *opt;
  return FWI_OK;
}

fwi_status fwi_plan_stats(const fwi_plan* plan, fwi_stats* out) {
  if (!plan || !out) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  *out = plan->stats;
  return FWI_OK;
}

fwi_status fwi_plan_estimate(const fwi_plan* plan, const fwi_geometry* geom, int gradient,
                             size_t* bytes) {
  if (!plan || !bytes) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  FWI_TRY(validate_geometry(plan, geom));
  Plan pl;
  FWI_TRY(choose_plan(plan, geom, true, gradient != 0, pl));
  *bytes = pl.bytes + tables_bound(plan, geom, pl) * 2;
  return FWI_OK;
}

void fwi_plan_destroy(fwi_plan* P) {
  if (!P) return;
  cudaSetDevice(P->device);
  if (P->st) cudaStreamSynchronize(P->st);
  else cudaDeviceSynchronize();
  cudaFree(P->arena);
  cudaFree(P->tab);
  cudaFree(P->spx);
  cudaFree(P->spy);
  cudaFree(P->spz);
  cudaFree(P->d_stats);
  cudaFree(P->d_flags);
  cudaFree(P->d_J);
  for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
  delete P;
}

fwi_status fwi_forward(fwi_plan* P, const fwi_model* model, const fwi_geometry* geom,
                       const float* wavelet, int nt, double dt, float* traces) {
  if (!P) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
  if (nt != P->nt || dt != P->dt) return fail(FWI_ERR_INVALID_ARG, "nt/dt differ from the plan's");
  if (!traces) return fail(FWI_ERR_INVALID_ARG, "traces is NULL");
  Call c;
  Carve tabC(nullptr);
  FWI_TRY(begin_call(P, model, geom, wavelet, false, c, tabC));
  const size_t fs = (size_t)P->L.fstride;
  const int B = c.pl.B;
  for (int shot0 = 0; shot0 < geom->nshots; shot0 += B) {
    const int nb = std::min(B, geom->nshots - shot0);
    Carve srcC = tabC;   // source tables of successive batches reuse the same space
    DevTable src;
    FWI_TRY(build_source_table(c, shot0, nb, srcC, src));
    float* A = c.W.U0;
    float* Bf = c.W.U1;
    CUDA_TRY(cudaMemsetAsync(A, 0, fs * nb * sizeof(float), P->st));
    CUDA_TRY(cudaMemsetAsync(Bf, 0, fs * nb * sizeof(float), P->st));
    FWI_TRY(forward_steps(c, nb, shot0, src, A, Bf, 0, P->nt - 1, nullptr, 0, true, 0, nullptr));
    FWI_TRY(final_sample(c, nb, A, P->nt - 1));
    cudaError_t e = launch_traces_out(c.W.D, traces, B, shot0, nb, geom->nrec, P->nt, P->d_flags, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
    // the next batch overwrites the source table: wait for this batch's launches to read it
    if (shot0 + B < geom->nshots) CUDA_TRY(cudaStreamSynchronize(P->st));
  }
  return finish_call(c);
}

fwi_status fwi_gradient(fwi_plan* P, const fwi_model* model, const fwi_geometry* geom,
                        const float* wavelet, const float* observed, double* misfit,
                        float* grad_m, float* traces_opt) {
  if (!P) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
  if (!observed || !misfit || !grad_m) return fail(FWI_ERR_INVALID_ARG, "observed, misfit or grad_m is NULL");
  Call c;
  Carve tabC(nullptr);
  FWI_TRY(begin_call(P, model, geom, wavelet, true, c, tabC));
  const size_t fs = (size_t)P->L.fstride;
  const int B = c.pl.B;
  const int nt = P->nt;
  const int K = c.pl.K;
  CUDA_TRY(cudaMemsetAsync(c.W.G, 0, fs * B * sizeof(float), P->st));
  int batch = 0;
  for (int shot0 = 0; shot0 < geom->nshots; shot0 += B, ++batch) {
    const int nb = std::min(B, geom->nshots - shot0);
    Carve srcC = tabC;
    DevTable src;
    FWI_TRY(build_source_table(c, shot0, nb, srcC, src));
    float* A = c.W.U0;
    float* Bf = c.W.U1;
    CUDA_TRY(cudaMemsetAsync(A, 0, fs * nb * sizeof(float), P->st));
    CUDA_TRY(cudaMemsetAsync(Bf, 0, fs * nb * sizeof(float), P->st));
    // forward sweep with history (K = 0) or checkpoints (K > 0)
    FWI_TRY(forward_steps(c, nb, shot0, src, A, Bf, 0, nt - 1, K == 0 ? c.W.H : nullptr, 0, true,
                          K, c.W.CK));
    FWI_TRY(final_sample(c, nb, A, nt - 1));
    // residual and misfit of this batch
    cudaError_t e = launch_misfit(c.W.D, observed, traces_opt, B, shot0, nb, geom->nrec, nt,
                                  c.W.partials, P->d_flags, c.W.npartials, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    e = launch_sum_partials(c.W.partials, misfit_blocks(nb, geom->nrec, nt), P->d_J + batch, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches += 2;
    // adjoint sweep: lambda^{nt-1} = lambda^{nt} = 0
    float* LA = (K == 0) ? c.W.U0 : c.W.F0;
    float* LB = (K == 0) ? c.W.U1 : c.W.F1;
    CUDA_TRY(cudaMemsetAsync(LA, 0, fs * nb * sizeof(float), P->st));
    CUDA_TRY(cudaMemsetAsync(LB, 0, fs * nb * sizeof(float), P->st));
    StepParams p = base_params(c);
    p.B = nb;
    p.inj_off = c.rec_tab.off;
    p.inj_loc = c.rec_tab.loc;
    p.inj_vidx = c.rec_tab.vidx;
    p.inj_w = c.rec_tab.w;
    p.vals = c.W.D;
    p.g = c.W.G;
    p.nrec = 0;
    int seg_lo = -1, seg_hi = -1;
    auto hist_at = [&](int n) -> float* {
      if (K == 0) return c.W.H + (size_t)n * fs * B;
      return c.W.H + (size_t)(n - seg_lo) * fs * B;
    };
    auto ensure_segment = [&](int n) -> fwi_status {
      if (K == 0 || (n >= seg_lo && n < seg_hi)) return FWI_OK;
      const int j = n / K;
      seg_lo = j * K;
      seg_hi = std::min(seg_lo + K, nt - 1);
      float* FA = c.W.U0;
      float* FB = c.W.U1;
      const float* ck = c.W.CK + 2 * (size_t)j * fs * B;
      CUDA_TRY(cudaMemcpyAsync(FA, ck, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
      CUDA_TRY(cudaMemcpyAsync(FB, ck + fs * B, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
      return forward_steps(c, nb, shot0, src, FA, FB, seg_lo, seg_hi, c.W.H, seg_lo, false, 0,
                           nullptr);
    };
    for (int k = nt - 1; k >= 1; --k) {
      p.image = (k <= nt - 2) ? 1 : 0;
      if (p.image) {
        FWI_TRY(ensure_segment(k));
        p.hist = hist_at(k);
      } else {
        p.hist = nullptr;
      }
      p.u = LA;
      p.up = LB;
      p.step_off = (long long)k * B * geom->nrec;
      FWI_TRY(launch_step(c, p, true));
      std::swap(LA, LB);
    }
    if (nt >= 2) {   // imaging term of lambda^0
      FWI_TRY(ensure_segment(0));
      e = launch_image_only(P->L, LA, hist_at(0), c.W.G, nb, P->st);
      if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
      c.launches++;
    }
    if (shot0 + B < geom->nshots) CUDA_TRY(cudaStreamSynchronize(P->st));
  }
  cudaError_t e = launch_grad_finalize(P->L, c.W.G, B, 1.0 / (P->dt * P->dt), grad_m, P->d_flags, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  c.launches++;
  std::vector<double> J(batch);
  CUDA_TRY(cudaMemcpyAsync(J.data(), P->d_J, sizeof(double) * batch, cudaMemcpyDeviceToHost, P->st));
  FWI_TRY(finish_call(c));
  double tot = 0.0;
  for (int i = 0; i < batch; ++i) tot += J[i];
  *misfit = tot;
  return FWI_OK;
}

}  // extern "C"

namespace fwi {

// Runs fwi_forward on a plan that lives on the stack and whose every device
// buffer is carved out of [base, base + bytes): no device allocation happens.
// Used by the fixed-scratch entry point (fwi_noalloc.cu).
fwi_status forward_in_buffer(const fwi_grid* grid, int nt, double dt, const fwi_model* model,
                             const fwi_geometry* geom, const float* wavelet, float* traces,
                             void* stream, char* base, size_t bytes, int device) {
  FWI_TRY(validate_grid(grid));
  if (nt < 1 || nt > (1 << 24)) return fail(FWI_ERR_INVALID_ARG, "nt must be in [1, 2^24]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FWI_ERR_INVALID_ARG, "dt must be positive");
  if (!traces) return fail(FWI_ERR_INVALID_ARG, "traces is NULL");
  if (!model || !model->vp) return fail(FWI_ERR_INVALID_ARG, "model or vp is NULL");
  fwi_plan P;
  P.grid = *grid;
  P.nt = nt;
  P.dt = dt;
  P.st = reinterpret_cast<cudaStream_t>(stream);
  P.device = device;
  P.c_ref = grid->c_ref;
  build_layout(&P);
  FWI_TRY(validate_geometry(&P, geom));
  constexpr int JCAP = 4096;
  Carve C(base);
  P.d_stats = C.take<unsigned int>(16);
  P.d_flags = C.take<int>(16);
  P.d_J = C.take<double>(JCAP);
  P.d_J_cap = JCAP;
  P.spx = C.take<float>(P.L.nx_r + 8);
  P.spy = C.take<float>(P.L.ny_r + 8);
  P.spz = C.take<float>(std::max(P.L.nz, 1) + 8);
  Plan all;
  all.B = geom->nshots;
  const size_t tab = align_up(tables_bound(&P, geom, all) * 2, 256);
  P.tab = C.take<char>(tab);
  P.tab_cap = tab;
  C.off = align_up(C.off, 256);
  if (C.off >= bytes)
    return fail(FWI_ERR_BUDGET, "tables need " + std::to_string(C.off) +
                                    " bytes, more than the static scratch of " +
                                    std::to_string(bytes) + " bytes");
  P.arena = base + C.off;
  P.arena_cap = bytes - C.off;
  P.budget = P.arena_cap;
  Plan pl;
  if (choose_plan(&P, geom, model->rho != nullptr, false, pl) != FWI_OK)
    return fail(FWI_ERR_BUDGET, "one shot of this grid needs more than the static scratch of " +
                                    std::to_string(bytes) + " bytes (use fwi_forward)");
  if ((geom->nshots + pl.B - 1) / pl.B > JCAP)
    return fail(FWI_ERR_BUDGET, "too many shot batches for the static scratch");
  if (P.c_ref > 0.0) FWI_TRY(build_sponge(&P));
  return fwi_forward(&P, model, geom, wavelet, nt, dt, traces);
}

}  // namespace fwi

namespace fwi {
// Sets the message fwi_last_error() returns on this thread.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace fwi
