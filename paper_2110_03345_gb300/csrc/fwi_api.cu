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

#include <cudaTypedefs.h>

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

constexpr double kPiD = 3.14159265358979323846;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round_up(int v, int a) { return (v + a - 1) / a * a; }

}  // namespace

namespace {
struct SavedGrad;
void delete_saved(SavedGrad* s);
}  // namespace

struct fwi_plan {
  fwi_grid grid{};
  int nt = 0;
  double dt = 0.0;
  size_t budget = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  int nsm = 152;            // SM count of the device
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
  SavedGrad* saved = nullptr;  // state kept by fwi_misfit_forward for fwi_misfit_backward
  bool fixed_memory = false;   // buffers supplied by the caller: never allocate
  ~fwi_plan() { delete_saved(saved); }
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

// Plan memory comes from the stream-ordered allocator on the plan's stream:
// unlike cudaMalloc/cudaFree it never synchronises the device, so plans on
// different streams (concurrent requests) do not serialise each other.
// Stream-ordered allocation from the device's default pool.  Freed plan
// workspaces stay reserved in the pool; when a request does not fit the
// pool's free pieces and the device, the unused reserve is returned to the
// device (trim) and the allocation retried once.
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t st, int device) {
  cudaError_t e = cudaMallocAsync(ptr, bytes, st);
  if (e == cudaSuccess) return e;
  cudaGetLastError();
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return e;
  cudaMemPoolTrimTo(pool, 0);
  return cudaMallocAsync(ptr, bytes, st);
}

// Device bytes a new workspace can take: free device memory plus the unused
// reserve of the default pool.
size_t device_available(int device) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
        reserved > used)
      fr += (size_t)(reserved - used);
  }
  cudaGetLastError();
  return fr;
}

fwi_status ensure_arena(fwi_plan* P, size_t bytes) {
  if (bytes <= P->arena_cap) return FWI_OK;
  if (P->fixed_memory)
    return fail(FWI_ERR_BUDGET, "workspace of " + std::to_string(bytes) + " bytes exceeds the fixed scratch");
  if (P->arena) {
    CUDA_TRY(cudaFreeAsync(P->arena, P->st));
    P->arena = nullptr;
    P->arena_cap = 0;
  }
  cudaError_t e = pool_alloc(reinterpret_cast<void**>(&P->arena), bytes, P->st, P->device);
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
  if (P->fixed_memory)
    return fail(FWI_ERR_BUDGET, "tables of " + std::to_string(bytes) + " bytes exceed the fixed scratch");
  if (P->tab) {
    CUDA_TRY(cudaFreeAsync(P->tab, P->st));
    P->tab = nullptr;
  }
  bytes = std::max(bytes, (size_t)1 << 20);
  CUDA_TRY(pool_alloc(reinterpret_cast<void**>(&P->tab), bytes, P->st, P->device));
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

TileGeo tile_geo(const fwi_plan* P, int tile, bool tma, bool x2 = false) {
  TileGeo T{};
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

HostTable bucket(const std::vector<Entry>& E_in, int nbuckets) {
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

// Floats per padded field of a grid: the layout build_layout gives it (x
// padded by OX and rounded to TILE_X plus 8, y by R each side and rounded to
// ROUND_Y, z by R each side, the field rounded to 64 floats).
long long padded_field_floats(const fwi_grid* g) {
  const long long R = g->order / 2;
  const long long nx = g->shape[g->ndim - 1], ny = g->shape[g->ndim - 2];
  const long long sx = OX + (nx + TILE_X - 1) / TILE_X * TILE_X + 8;
  const long long rows = R + (ny + ROUND_Y - 1) / ROUND_Y * ROUND_Y + R;
  const long long planes = g->ndim == 3 ? g->shape[0] + 2 * R : 1;
  return (sx * rows * planes + 63) / 64 * 64;
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
  // The second-fastest axis is split over grid.y (at least 8 rows per CTA),
  // which CUDA limits to 65535 blocks.
  if (g->shape[g->ndim - 2] > 8LL * 65535)
    return fail(FWI_ERR_INVALID_ARG, "shape out of range: the second-fastest axis exceeds 524280 points");
  // In-field offsets (receiver sampling tables, tile-local arithmetic) are
  // 32-bit: a padded field must hold fewer than 2^31 floats.
  if (padded_field_floats(g) > 0x7fffffffLL)
    return fail(FWI_ERR_INVALID_ARG, "grid too large: a padded field exceeds 2^31 - 1 floats");
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
  L.fstride = (long long)align_up((size_t)(L.sxy * L.planes), 64);   // = padded_field_floats
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
    if (!*dst[a]) CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(dst[a]), v.size() * sizeof(float), P->st));
    CUDA_TRY(cudaMemcpyAsync(*dst[a], v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice, P->st));
    CUDA_TRY(cudaStreamSynchronize(P->st));   // v is a host temporary
  }
  P->sponge_ready = true;
  return FWI_OK;
}

fwi_status validate_geometry(const fwi_plan* P, const fwi_geometry* g) {
  if (!g) return fail(FWI_ERR_INVALID_ARG, "geometry is NULL");
  if (g->nshots < 1 || g->nsrc < 1 || g->nrec < 1)
    return fail(FWI_ERR_INVALID_ARG, "nshots, nsrc and nrec must be >= 1");
  if (!g->src_xyz || !g->rec_xyz) return fail(FWI_ERR_INVALID_ARG, "coordinates are NULL");
  if ((long long)g->nshots * g->nsrc > (1LL << 24) || g->nrec > (1 << 20))
    return fail(FWI_ERR_INVALID_ARG, "too many sources (2^24) or receivers (2^20)");
  // wavelet and trace samples are addressed with 32-bit indices
  if ((long long)g->nshots * g->nsrc * P->nt > 0x7fffffffLL ||
      (long long)g->nshots * g->nrec * P->nt > 0x7fffffffLL)
    return fail(FWI_ERR_INVALID_ARG,
                "the wavelet or trace array would hold 2^31 samples or more: split the shots over calls");
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
  int tile = 0;         // resolved variant id (as in fwi_options.tile, never 0)
  int shape = 0;        // tile shape 0..3
  bool tma = false;     // TMA-staged kernels (2D: shots looped inside a CTA)
  bool x2 = false;      // 3D: two x points per thread (variants 9-12)
  int S = 1;            // shots per CTA; gradient slot of shot s is s / S
  bool split = false;   // forward and adjoint in separate calls: keep every batch's state
  int nbatches = 1;
  size_t bytes = 0;
};

// Resolve fwi_options.tile: 0 selects the default variant.
bool resolve_tile(const fwi_plan* P, int t, int* id, int* shape, bool* tma, bool* x2 = nullptr) {
  if (x2) *x2 = false;
  if (P->grid.ndim == 2) {
    if (t == 0) t = 6;   // TMA-staged, one row per thread, 128 x 16 tiles
    if (t < 1 || t > 2 * NUM_TILE2) return false;
    *tma = t > NUM_TILE2;
    *shape = (t - 1) % NUM_TILE2;
  } else {
    if (t == 0) t = 12;  // TMA-staged plane ring, two points per thread, 64 x 8 columns, 32-plane chunks
    if (t < 1 || t > 3 * NUM_TILE3) return false;
    *tma = t > NUM_TILE3;
    if (x2) *x2 = t > 2 * NUM_TILE3;
    *shape = (t - 1) % NUM_TILE3;
  }
  *id = t;
  return true;
}

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

// Split gradient: bytes kept per shot between the two calls (checkpoints or
// history, and the residual traces), and the per-slot working set.
size_t persist_bytes_per_shot(const fwi_plan* P, const fwi_geometry* g, int K) {
  const size_t f = align_up(field_bytes(P), 256);
  const size_t traces = (size_t)P->nt * g->nrec * sizeof(float);
  if (K == 0) return (size_t)std::max(P->nt - 1, 1) * f + traces;
  const int nck = (P->nt - 2) / K + 1;
  return 2 * (size_t)nck * f + traces;
}

size_t split_slot_bytes(const fwi_plan* P, int K) {
  const size_t f = align_up(field_bytes(P), 256);
  return 5 * f + (K ? (size_t)K * f : 0) + 4096;
}

size_t fixed_bytes(const fwi_plan* P, const fwi_geometry* g, bool vd, int B) {
  const size_t misfit = align_up((size_t)misfit_blocks(B, g->nrec, P->nt) * 8, 256);
  return model_bytes(P, vd) + misfit + (4u << 20);
}

fwi_status choose_plan(const fwi_plan* P, const fwi_geometry* g, bool vd, bool grad, Plan& out,
                       bool split = false) {
  const int ns = g->nshots;
  const size_t budget = P->budget;
  const int K_auto = std::max(2, (int)std::ceil(std::sqrt(2.0 * std::max(P->nt, 2))));
  const long long N = (long long)P->L.nx * P->L.ny * P->L.nz;
  const int B_fill = (int)std::max(1LL, (8LL << 20) / std::max(N, 1LL));  // slots that fill the GPU
  auto fit = [&](int K) {
    size_t fixed = fixed_bytes(P, g, vd, ns);
    size_t per = slot_bytes(P, g, grad, K);
    if (split) {
      // nbatches * B <= ns + B - 1 shots of kept state
      const size_t keep = persist_bytes_per_shot(P, g, K);
      fixed += (size_t)ns * keep;
      per = split_slot_bytes(P, K) + keep;
    }
    if (budget <= fixed) return 0;
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
  if (!resolve_tile(P, P->opt.tile, &out.tile, &out.shape, &out.tma, &out.x2))
    return fail(FWI_ERR_INVALID_ARG, "tile variant out of range");
  // slots x z chunks go on grid.z, which CUDA limits to 65535 blocks
  B = std::min(B, std::max(1, 65535 / std::max(1, tile_geo(P, out.shape, out.tma, out.x2).nzc)));
  // equal batches: the same number of batches, none left nearly empty
  // (16 shots at 15 per batch run as 8 + 8, not 15 + 1)
  B = (ns + (ns + B - 1) / B - 1) / ((ns + B - 1) / B);
  out.B = B;
  out.K = K;
  out.nck = K ? (P->nt - 2) / K + 1 : 0;
  out.gradient = grad;
  out.split = split;
  out.nbatches = (ns + B - 1) / B;
  out.S = 1;
  if (out.tma && P->grid.ndim == 2) {   // the 3D kernels take one shot per CTA
    if (P->opt.shots_per_cta > 0) {
      out.S = std::min(P->opt.shots_per_cta, B);
    } else {
      // six shots share a tile's model loads and gradient update; at least
      // four waves of CTAs (two resident per SM) keep the SMs balanced
      const int T = tile_geo(P, out.shape, true).ntiles();
      int S = std::min(B, 6);
      while (S > 1 && (long long)T * ((B + S - 1) / S) < 8LL * P->nsm) --S;
      out.S = S;
    }
  }
  out.bytes = fixed_bytes(P, g, vd, B) + (size_t)B * slot_bytes(P, g, grad, K);
  if (split)
    out.bytes = fixed_bytes(P, g, vd, B) + (size_t)B * split_slot_bytes(P, K) +
                (size_t)out.nbatches * B * persist_bytes_per_shot(P, g, K) + (4u << 20);
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
  const size_t nbk = pl.split ? (size_t)pl.nbatches : 1;   // batches whose state is kept
  W.D = C.take<float>((size_t)P->nt * B * g->nrec * nbk);
  if (pl.gradient) {
    W.G = C.take<float>(fs * B);
    if (pl.K == 0) {
      W.H = C.take<float>(fs * B * (size_t)std::max(P->nt - 1, 1) * nbk);
    } else {
      W.F0 = C.take<float>(fs * B);
      W.F1 = C.take<float>(fs * B);
      W.CK = C.take<float>(fs * B * 2 * (size_t)pl.nck * nbk);
      W.H = C.take<float>(fs * B * (size_t)pl.K);
    }
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// 3D tensor map over nslots padded 2D fields: dims (x = sx, y = rows, slot),
// box = one tile plus its halo of one slot.
fwi_status make_tensor_map(const fwi_plan* P, const float* base, int nslots, int shape,
                           CUtensorMap* out) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  int bx = 0, by = 0;
  tma_box2d(P->R, shape, &bx, &by);
  const cuuint64_t dims[3] = {(cuuint64_t)P->L.sx, (cuuint64_t)P->L.rows, (cuuint64_t)nslots};
  const cuuint64_t strides[2] = {(cuuint64_t)P->L.sx * sizeof(float),
                                 (cuuint64_t)P->L.fstride * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return FWI_OK;
}

// 4D tensor map over nslots padded 3D fields: dims (x, y, z, slot); box = a
// 48-float-wide (80 for the two-point kernels) x-y tile (16-byte aligned
// start) with its y halo, one plane.
fwi_status make_tensor_map_3d(const fwi_plan* P, const float* base, int nslots, int shape,
                              bool x2, CUtensorMap* out) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[4] = {(cuuint64_t)P->L.sx, (cuuint64_t)P->L.rows, (cuuint64_t)P->L.planes,
                              (cuuint64_t)nslots};
  const cuuint64_t strides[3] = {(cuuint64_t)P->L.sx * sizeof(float),
                                 (cuuint64_t)P->L.sxy * sizeof(float),
                                 (cuuint64_t)P->L.fstride * sizeof(float)};
  const cuuint32_t box[4] = {x2 ? 80u : 48u, (cuuint32_t)tma_box3d_rows(P->R, shape), 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled (3D) failed with code " + std::to_string((int)r));
  return FWI_OK;
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
  float* D = nullptr; // trace / residual buffer [nt][B][nrec] of the current batch
  int ncorner = 4;
  struct MapEnt {
    const float* base;
    CUtensorMap map;
  };
  std::vector<MapEnt> maps;   // TMA descriptors of the wavefield buffers
  int64_t launches = 0;
  int64_t fwd_launches = 0, adj_launches = 0;
  int64_t fwd_points = 0, adj_points = 0;
  int64_t fwd_timed = 0, adj_timed = 0;   // launches that carried events
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
  for (int a = 0; a < 3; ++a) {
    const bool on = a < P->grid.ndim;
    p.ih2[a] = on ? (float)(1.0 / (P->h[a] * P->h[a])) : 0.f;
    p.ih1[a] = on ? (float)(1.0 / P->h[a]) : 0.f;
  }
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
  const int by = (c.P->grid.ndim == 3) ? tile3_variant(c.pl.shape).by
                 : c.pl.tma ? tile2_tma_variant(c.pl.shape).by : tile2_variant(c.pl.shape).by;
  const int ctas_z = (B + c.pl.S - 1) / c.pl.S;
  return (long long)c.T.ntiles() * ctas_z * 32 * by;
}

const CUtensorMap* find_map(const Call& c, const float* base) {
  for (const auto& m : c.maps)
    if (m.base == base) return &m.map;
  return nullptr;
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
  const bool prof = P->opt.profile > 0 &&
                    (c.fwd_launches + c.adj_launches) % P->opt.profile == 0;
  p.flags = P->d_flags + 1;
  p.S = c.pl.S;
  const CUtensorMap* map = nullptr;
  if (c.pl.tma) {
    map = find_map(c, p.u);
    if (!map) return fail(FWI_ERR_INVALID_ARG, "internal: no tensor map for the wavefield buffer");
  }
  if (prof) FWI_TRY(record_event(P, adj ? 1 : 0));
  cudaError_t e;
  if (P->grid.ndim == 3 && c.pl.tma) {
    const CUtensorMap* bxm = c.vd ? find_map(c, c.W.bx) : map;
    const CUtensorMap* bym = c.vd ? find_map(c, c.W.by) : map;
    if (!bxm || !bym) return fail(FWI_ERR_INVALID_ARG, "internal: no tensor map for b_x / b_y");
    e = c.pl.x2 ? launch_step3d_x2(p, *map, *bxm, *bym, P->R, c.vd, adj, c.pl.shape, P->st)
                : launch_step3d_tma(p, *map, *bxm, *bym, P->R, c.vd, adj, c.pl.shape, P->st);
  } else if (P->grid.ndim == 3) e = launch_step3d(p, P->R, c.vd, adj, c.pl.shape, P->st);
  else if (c.pl.tma) e = launch_step2d_tma(p, *map, P->R, c.vd, adj, c.pl.shape, P->st);
  else e = launch_step2d(p, P->R, c.vd, adj, c.pl.shape, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("stencil launch: ") + cudaGetErrorString(e));
  if (prof) {
    FWI_TRY(record_event(P, adj ? 1 : 0));
    if (adj) c.adj_timed++;
    else c.fwd_timed++;
  }
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
  p.smp_out = c.D;
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
  p.smp_out = c.D;
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
  c.T = tile_geo(P, c.pl.shape, c.pl.tma, c.pl.x2);
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
  const TileGeo T = tile_geo(P, pl.shape, pl.tma, pl.x2);
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
  if (m->param != FWI_PARAM_VP && m->param != FWI_PARAM_M)
    return fail(FWI_ERR_INVALID_ARG, "model param must be FWI_PARAM_VP or FWI_PARAM_M");
  cudaError_t e = launch_model_prep(P->L, m->vp, m->rho, P->dt, m->param, c.W.kf,
                                    c.vd ? c.W.lnr : nullptr, P->d_stats, P->st);
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
                      const float* wavelet, bool grad, Call& c, Carve& tabC, bool split = false) {
  if (!model || !model->vp) return fail(FWI_ERR_INVALID_ARG, "model or vp is NULL");
  if (!wavelet) return fail(FWI_ERR_INVALID_ARG, "wavelet is NULL");
  FWI_TRY(validate_geometry(P, geom));
  CUDA_TRY(cudaSetDevice(P->device));
  c.P = P;
  c.model = model;
  c.geom = geom;
  c.wavelet = wavelet;
  c.vd = model->rho != nullptr;
  if (P->saved) {   // any new call drops the state of a pending split gradient
    delete_saved(P->saved);
    P->saved = nullptr;
  }
  FWI_TRY(choose_plan(P, geom, c.vd, grad, c.pl, split));
  FWI_TRY(ensure_arena(P, c.pl.bytes));
  Carve C(P->arena);
  carve_work(P, c.pl, geom, c.vd, C, c.W);
  if (C.off > P->arena_cap) return fail(FWI_ERR_BUDGET, "workspace carve exceeds allocation");
  if (c.pl.tma) {
    const bool three = P->grid.ndim == 3;
    for (float* buf : {c.W.U0, c.W.U1, c.W.F0, c.W.F1}) {
      if (!buf) continue;
      Call::MapEnt m{buf, {}};
      if (three) FWI_TRY(make_tensor_map_3d(P, buf, c.pl.B, c.pl.shape, c.pl.x2, &m.map));
      else FWI_TRY(make_tensor_map(P, buf, c.pl.B, c.pl.shape, &m.map));
      c.maps.push_back(m);
    }
    if (three && c.vd) {
      for (float* buf : {c.W.bx, c.W.by}) {
        Call::MapEnt m{buf, {}};
        FWI_TRY(make_tensor_map_3d(P, buf, 1, c.pl.shape, c.pl.x2, &m.map));
        c.maps.push_back(m);
      }
    }
  }
  FWI_TRY(ensure_tab(P, tables_bound(P, geom, c.pl) * 2));
  tabC = Carve(P->tab);
  const int nbatches = (geom->nshots + c.pl.B - 1) / c.pl.B;
  if (nbatches > P->d_J_cap) {
    if (P->fixed_memory) return fail(FWI_ERR_BUDGET, "too many shot batches for the fixed scratch");
    if (P->d_J) CUDA_TRY(cudaFreeAsync(P->d_J, P->st));
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&P->d_J), sizeof(double) * nbatches, P->st));
    P->d_J_cap = nbatches;
  }
  CUDA_TRY(cudaMemsetAsync(P->d_flags, 0, sizeof(int) * 4, P->st));
  P->ev_used = 0;
  c.D = c.W.D;
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
  s.fwd_timed = c.fwd_timed;
  s.adj_timed = c.adj_timed;
  s.updates = c.fwd_points + c.adj_points;
  s.fwd_ms = s.adj_ms = 0.0;
  for (size_t i = 0; i + 1 < P->ev_used; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]));
    if (P->ev_kind[i] == 0) s.fwd_ms += ms;
    else s.adj_ms += ms;
  }
  if (flags[1] & 2) return fail(FWI_ERR_TIMEOUT, "a bounded wait on a TMA copy timed out");
  if (flags[0]) return fail(FWI_ERR_NONFINITE, "non-finite values in the result (unstable run?)");
  return FWI_OK;
}

// State kept between fwi_misfit_forward and fwi_misfit_backward.
struct SavedGrad {
  Call c;
  Carve tabC{nullptr};
  std::vector<double> src, rec;
  fwi_geometry geom{};
  fwi_model model{};
  int nbatches = 0;
  double J = 0.0;
};

void delete_saved(SavedGrad* s) { delete s; }

// Pointers of batch j's kept state: traces/residuals, checkpoints, history.
struct BatchBufs {
  float* D;
  float* CK;
  float* H;
};

BatchBufs batch_bufs(const Call& c, int j) {
  const size_t fs = (size_t)c.P->L.fstride;
  const size_t B = (size_t)c.pl.B;
  const size_t k = c.pl.split ? (size_t)j : 0;
  const int nt = c.P->nt;
  BatchBufs b;
  b.D = c.W.D + k * (size_t)nt * B * c.geom->nrec;
  b.CK = c.W.CK ? c.W.CK + k * fs * B * 2 * (size_t)c.pl.nck : nullptr;
  b.H = (c.pl.K == 0) ? c.W.H + k * fs * B * (size_t)std::max(nt - 1, 1) : c.W.H;
  return b;
}

// Forward sweep of batch j (history or checkpoints), last trace sample,
// residual and misfit of the batch (into d_J[j]).
fwi_status gradient_forward_batch(Call& c, int j, int shot0, int nb, const DevTable& src,
                                  const float* observed, float* traces_opt) {
  fwi_plan* P = c.P;
  const size_t fs = (size_t)P->L.fstride;
  const int nt = P->nt;
  const int K = c.pl.K;
  const BatchBufs bb = batch_bufs(c, j);
  c.D = bb.D;
  float* A = c.W.U0;
  float* Bf = c.W.U1;
  CUDA_TRY(cudaMemsetAsync(A, 0, fs * nb * sizeof(float), P->st));
  CUDA_TRY(cudaMemsetAsync(Bf, 0, fs * nb * sizeof(float), P->st));
  FWI_TRY(forward_steps(c, nb, shot0, src, A, Bf, 0, nt - 1, K == 0 ? bb.H : nullptr, 0, true,
                        K, bb.CK));
  FWI_TRY(final_sample(c, nb, A, nt - 1));
  cudaError_t e = launch_misfit(c.D, observed, traces_opt, c.pl.B, shot0, nb, c.geom->nrec, nt,
                                c.W.partials, P->d_flags, c.W.npartials, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  e = launch_sum_partials(c.W.partials, misfit_blocks(nb, c.geom->nrec, nt), P->d_J + j, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  c.launches += 2;
  return FWI_OK;
}

// Adjoint sweep of batch j with the imaging condition, from the kept history
// or by recomputing each checkpoint segment; accumulates into the slots of G.
fwi_status gradient_adjoint_batch(Call& c, int j, int shot0, int nb, const DevTable& src) {
  fwi_plan* P = c.P;
  const size_t fs = (size_t)P->L.fstride;
  const int B = c.pl.B;
  const int nt = P->nt;
  const int K = c.pl.K;
  const BatchBufs bb = batch_bufs(c, j);
  c.D = bb.D;
  // lambda^{nt-1} = lambda^{nt} = 0
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
  p.vals = c.D;
  p.g = c.W.G;
  p.nrec = 0;
  int seg_lo = -1, seg_hi = -1;
  auto hist_at = [&](int n) -> float* {
    if (K == 0) return bb.H + (size_t)n * fs * B;
    return bb.H + (size_t)(n - seg_lo) * fs * B;
  };
  auto ensure_segment = [&](int n) -> fwi_status {
    if (K == 0 || (n >= seg_lo && n < seg_hi)) return FWI_OK;
    const int js = n / K;
    seg_lo = js * K;
    seg_hi = std::min(seg_lo + K, nt - 1);
    float* FA = c.W.U0;
    float* FB = c.W.U1;
    const float* ck = bb.CK + 2 * (size_t)js * fs * B;
    CUDA_TRY(cudaMemcpyAsync(FA, ck, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
    CUDA_TRY(cudaMemcpyAsync(FB, ck + fs * B, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
    return forward_steps(c, nb, shot0, src, FA, FB, seg_lo, seg_hi, bb.H, seg_lo, false, 0, nullptr);
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
    p.step_off = (long long)k * B * c.geom->nrec;
    FWI_TRY(launch_step(c, p, true));
    std::swap(LA, LB);
  }
  if (nt >= 2) {   // imaging term of lambda^0
    FWI_TRY(ensure_segment(0));
    cudaError_t e = launch_image_only(P->L, LA, hist_at(0), c.W.G, nb, c.pl.S, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
  }
  return FWI_OK;
}

// Sum the gradient slots into grad_m (scaled by 1/dt^2), read the misfit of
// `batches` batches (0: none) and finish the call.
fwi_status gradient_finish(Call& c, int batches, double* misfit, float* grad_m) {
  fwi_plan* P = c.P;
  const int G = (c.pl.B + c.pl.S - 1) / c.pl.S;   // gradient slots in use
  cudaError_t e = launch_grad_finalize(P->L, c.W.G, G, 1.0 / (P->dt * P->dt), grad_m, P->d_flags, P->st);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  c.launches++;
  std::vector<double> J(std::max(batches, 1));
  if (batches > 0)
    CUDA_TRY(cudaMemcpyAsync(J.data(), P->d_J, sizeof(double) * batches, cudaMemcpyDeviceToHost, P->st));
  FWI_TRY(finish_call(c));
  double tot = 0.0;
  for (int i = 0; i < batches; ++i) tot += J[i];
  if (batches > 0) *misfit = tot;
  return FWI_OK;
}

}  // namespace

extern "C" {

const char* fwi_last_error(void) { return g_err.c_str(); }

fwi_status fwi_mem_available(size_t* bytes) {
  if (!bytes) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_CUDA, "no CUDA device");
  }
  *bytes = device_available(dev);
  return FWI_OK;
}

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
  // Kaiser-windowed sinc: per axis the 2r nodes floor(x)-r+1 .. floor(x)+r
  // with w = I0(b sqrt(1 - (d/r)^2)) / I0(b) * sin(pi d) / (pi d), d = i - x;
  // the point weights are the products over the axes.
  constexpr int r = FWI_SINC_RADIUS;
  constexpr double b = FWI_SINC_KAISER_B;
  auto bessel_i0 = [](double x) {          // power series sum_k ((x/2)^k / k!)^2
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200 && term > 1e-18 * sum; ++k) {
      term *= (x / (2.0 * k)) * (x / (2.0 * k));
      sum += term;
    }
    return sum;
  };
  const double i0b = bessel_i0(b);
  int first[3] = {0, 0, 0};
  double w1[3][2 * FWI_SINC_RADIUS];
  int total = 1;
  for (int d = 0; d < nd; ++d) {
    const double x = xyz[d] / grid->spacing[d];
    const long long f = (long long)std::floor(x);
    if (f - r + 1 < 0 || f + r > grid->shape[d] - 1)
      return fail(FWI_ERR_INVALID_ARG, "fwi_point_weights: a sinc point must lie r - 1 nodes inside every face");
    first[d] = (int)(f - r + 1);
    for (int j = 0; j < 2 * r; ++j) {
      const double dd = (double)(first[d] + j) - x;
      const double q = 1.0 - (dd / r) * (dd / r);
      const double win = std::fabs(dd) <= r ? bessel_i0(b * std::sqrt(q > 0.0 ? q : 0.0)) / i0b : 0.0;
      const double sn = dd == 0.0 ? 1.0 : std::sin(kPiD * dd) / (kPiD * dd);
      w1[d][j] = win * sn;
    }
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
  fr = device_available(P->device);   // free memory plus the pool's unused reserve
  P->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  if (cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
    cudaGetLastError();
    P->nsm = 152;
  }
  {
    // keep freed plan memory cached in the default pool (no return to the OS
    // between requests); this is a per-process allocator setting
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, P->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  if (cudaMallocAsync(reinterpret_cast<void**>(&P->d_stats), 64, P->st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&P->d_flags), 64, P->st) != cudaSuccess)
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
  if (opt->profile < 0) return fail(FWI_ERR_INVALID_ARG, "profile must be >= 0");
  if (opt->use_graphs != 0) return fail(FWI_ERR_UNSUPPORTED, "use_graphs is reserved and must be 0");
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
  for (void* q : {(void*)P->arena, (void*)P->tab, (void*)P->spx, (void*)P->spy, (void*)P->spz,
                  (void*)P->d_stats, (void*)P->d_flags, (void*)P->d_J})
    if (q) cudaFreeAsync(q, P->st);
  cudaStreamSynchronize(P->st);
  cudaGetLastError();
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
  CUDA_TRY(cudaMemsetAsync(c.W.G, 0, fs * c.pl.B * sizeof(float), P->st));
  int batch = 0;
  for (int shot0 = 0; shot0 < geom->nshots; shot0 += c.pl.B, ++batch) {
    const int nb = std::min(c.pl.B, geom->nshots - shot0);
    Carve srcC = tabC;
    DevTable src;
    FWI_TRY(build_source_table(c, shot0, nb, srcC, src));
    FWI_TRY(gradient_forward_batch(c, batch, shot0, nb, src, observed, traces_opt));
    FWI_TRY(gradient_adjoint_batch(c, batch, shot0, nb, src));
    if (shot0 + c.pl.B < geom->nshots) CUDA_TRY(cudaStreamSynchronize(P->st));
  }
  return gradient_finish(c, batch, misfit, grad_m);
}

fwi_status fwi_misfit_forward(fwi_plan* P, const fwi_model* model, const fwi_geometry* geom,
                              const float* wavelet, const float* observed, double* misfit,
                              float* traces_opt) {
  if (!P) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
  if (!observed || !misfit) return fail(FWI_ERR_INVALID_ARG, "observed or misfit is NULL");
  if (!model || !geom) return fail(FWI_ERR_INVALID_ARG, "model or geometry is NULL");
  // keep host copies of the geometry; device arrays stay the caller's
  SavedGrad* S = new SavedGrad();
  S->src.assign(geom->src_xyz, geom->src_xyz + (size_t)geom->nshots * geom->nsrc * P->grid.ndim);
  S->rec.assign(geom->rec_xyz, geom->rec_xyz + (size_t)geom->nrec * P->grid.ndim);
  S->geom = *geom;
  S->geom.src_xyz = S->src.data();
  S->geom.rec_xyz = S->rec.data();
  S->model = *model;
  Call& c = S->c;
  fwi_status st = begin_call(P, &S->model, &S->geom, wavelet, true, c, S->tabC, true);
  if (st != FWI_OK) {
    delete_saved(S);
    return st;
  }
  int batch = 0;
  for (int shot0 = 0; shot0 < geom->nshots && st == FWI_OK; shot0 += c.pl.B, ++batch) {
    const int nb = std::min(c.pl.B, geom->nshots - shot0);
    Carve srcC = S->tabC;
    DevTable src;
    st = build_source_table(c, shot0, nb, srcC, src);
    if (st == FWI_OK) st = gradient_forward_batch(c, batch, shot0, nb, src, observed, traces_opt);
    if (st == FWI_OK && shot0 + c.pl.B < geom->nshots) {
      cudaError_t e = cudaStreamSynchronize(P->st);
      if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  std::vector<double> J(batch);
  if (st == FWI_OK) {
    cudaError_t e = cudaMemcpyAsync(J.data(), P->d_J, sizeof(double) * batch, cudaMemcpyDeviceToHost, P->st);
    if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  }
  if (st == FWI_OK) st = finish_call(c);
  if (st != FWI_OK) {
    delete_saved(S);
    return st;
  }
  double tot = 0.0;
  for (int i = 0; i < batch; ++i) tot += J[i];
  *misfit = tot;
  S->nbatches = batch;
  S->J = tot;
  P->saved = S;
  return FWI_OK;
}

fwi_status fwi_misfit_backward(fwi_plan* P, float* grad_m) {
  if (!P || !grad_m) return fail(FWI_ERR_INVALID_ARG, "plan or grad_m is NULL");
  SavedGrad* S = P->saved;
  if (!S) return fail(FWI_ERR_INVALID_ARG, "no pending fwi_misfit_forward on this plan");
  P->saved = nullptr;   // the state is used once
  Call& c = S->c;
  CUDA_TRY(cudaSetDevice(P->device));
  const size_t fs = (size_t)P->L.fstride;
  c.launches = c.fwd_launches = c.adj_launches = c.fwd_points = c.adj_points = 0;
  P->ev_used = 0;
  fwi_status st = FWI_OK;
  cudaError_t e = cudaMemsetAsync(c.W.G, 0, fs * c.pl.B * sizeof(float), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->d_flags, 0, sizeof(int) * 4, P->st);
  if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  int batch = 0;
  for (int shot0 = 0; shot0 < S->geom.nshots && st == FWI_OK; shot0 += c.pl.B, ++batch) {
    const int nb = std::min(c.pl.B, S->geom.nshots - shot0);
    Carve srcC = S->tabC;
    DevTable src;
    st = build_source_table(c, shot0, nb, srcC, src);
    if (st == FWI_OK) st = gradient_adjoint_batch(c, batch, shot0, nb, src);
    if (st == FWI_OK && shot0 + c.pl.B < S->geom.nshots) {
      e = cudaStreamSynchronize(P->st);
      if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  double J = 0.0;
  if (st == FWI_OK) st = gradient_finish(c, 0, &J, grad_m);
  delete_saved(S);
  return st;
}

}  // extern "C"

#define FWI_TRY_B(call)              \
  do {                               \
    fwi_status s_ = (call);          \
    if (s_ != FWI_OK) return bail(s_); \
  } while (0)

#define CUDA_TRY_B(call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bail(fail(FWI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)));   \
  } while (0)

// ---------------------------------------------------------------------------
// Uneven batches of independent 2D problems (forward modelling).
// ---------------------------------------------------------------------------
namespace {

struct BatchProblem {
  fwi_plan* P = nullptr;
  Call c;
  Carve tabC{nullptr};
  DevTable src;
  fwi_problem prob{};
  std::vector<double> srcxyz, recxyz;
};

}  // namespace

struct fwi_batch {
  std::vector<BatchProblem*> items;   // sorted by nt, longest first
  cudaStream_t st = nullptr;          // the caller's stream
  cudaStream_t ws = nullptr;          // internal non-blocking stream the runs (and the capture) use
  cudaEvent_t ready = nullptr;
  int device = 0;
  int R = 4;
  bool vd = false;
  bool tma = true;      // TMA-staged multi-problem kernel (else shared-memory staged)
  int shape = 0;        // tile shape of the batch's kernels
  bool uniform_w = false;   // every problem has the same stencil weights
  AxisW w[2] = {};          // {x, y} weights when uniform_w
  MultiDesc* d_desc = nullptr;
  MultiUnit* d_units = nullptr;
  std::vector<int> active_units;      // units of the problems still running at step n
  int max_steps = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  fwi_batch_stats stats{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~fwi_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(d_desc);
    cudaFree(d_units);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ready) cudaEventDestroy(ready);
    if (ws) cudaStreamDestroy(ws);
    for (BatchProblem* b : items) {
      fwi_plan_destroy(b->P);
      delete b;
    }
  }
};

namespace {

// Every step of every problem (and the final sampling / trace transposition)
// enqueued on b->st; captured into a graph when b->use_graph.
fwi_status batch_enqueue(fwi_batch* b) {
  int64_t launches = 0, updates = 0;
  for (int n = 0; n < b->max_steps; ++n) {
    cudaError_t e = b->tma ? launch_step2d_tma_multi(b->d_desc, b->d_units, b->active_units[n], n,
                                                     b->R, b->vd, b->shape,
                                                     b->uniform_w ? b->w : nullptr, b->ws)
                           : launch_step2d_multi(b->d_desc, b->d_units, b->active_units[n], n,
                                                 b->R, b->vd, b->ws);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("multi-problem step: ") + cudaGetErrorString(e));
    ++launches;
  }
  for (BatchProblem* it : b->items) {
    Call& c = it->c;
    const int nt = it->prob.nt;
    const int ns = it->prob.geom.nshots;
    float* last = ((nt - 1) & 1) ? c.W.U1 : c.W.U0;   // u^{nt-1}
    StepParams p = base_params(c);
    p.B = ns;
    p.u = last;
    p.smp_node = c.smp_node;
    p.smp_w = c.smp_w;
    p.smp_out = c.W.D;
    p.nrec = it->prob.geom.nrec;
    p.smp_off = (long long)(nt - 1) * c.pl.B * it->prob.geom.nrec;
    cudaError_t e = launch_sample(p, b->ws);
    if (e == cudaSuccess)
      e = launch_traces_out(c.W.D, it->prob.traces, c.pl.B, 0, ns, it->prob.geom.nrec, nt,
                            it->P->d_flags, b->ws);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    launches += 2;
    updates += (int64_t)ns * it->P->L.nx * it->P->L.ny * (nt - 1);
  }
  b->stats.launches = launches;
  b->stats.updates = updates;
  return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_batch_create(fwi_batch** out, int nprob, const fwi_problem* probs,
                            const fwi_options* opt, size_t hbm_budget_bytes, void* stream,
                            int use_graph) {
  if (!out || !probs || nprob < 1) return fail(FWI_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  fwi_batch* b = new fwi_batch();
  b->st = reinterpret_cast<cudaStream_t>(stream);
  b->use_graph = use_graph != 0;
  auto bail = [&](fwi_status s) { delete b; return s; };
  if (cudaGetDevice(&b->device) != cudaSuccess) return bail(fail(FWI_ERR_CUDA, "no CUDA device"));
  size_t used = 0;
  for (int i = 0; i < nprob; ++i) {
    const fwi_problem& pr = probs[i];
    if (pr.grid.ndim != 2) return bail(fail(FWI_ERR_UNSUPPORTED, "batches hold 2D problems"));
    if (i == 0) {
      b->R = pr.grid.order / 2;
      b->vd = pr.model.rho != nullptr;
    } else if (pr.grid.order / 2 != b->R || (pr.model.rho != nullptr) != b->vd) {
      return bail(fail(FWI_ERR_UNSUPPORTED, "a batch shares one stencil order and density mode"));
    }
    if (!pr.traces || !pr.wavelet) return bail(fail(FWI_ERR_INVALID_ARG, "problem arrays are NULL"));
    BatchProblem* it = new BatchProblem();
    b->items.push_back(it);
    it->prob = pr;
    if (!pr.geom.src_xyz || !pr.geom.rec_xyz) return bail(fail(FWI_ERR_INVALID_ARG, "coordinates are NULL"));
    it->srcxyz.assign(pr.geom.src_xyz, pr.geom.src_xyz + (size_t)pr.geom.nshots * pr.geom.nsrc * 2);
    it->recxyz.assign(pr.geom.rec_xyz, pr.geom.rec_xyz + (size_t)pr.geom.nrec * 2);
    it->prob.geom.src_xyz = it->srcxyz.data();
    it->prob.geom.rec_xyz = it->recxyz.data();
    const size_t left = hbm_budget_bytes ? (hbm_budget_bytes > used ? hbm_budget_bytes - used : 1) : 0;
    FWI_TRY_B(fwi_plan_create(&it->P, &pr.grid, pr.nt, pr.dt, left, stream));
    fwi_options o{};
    o.batch = pr.geom.nshots;   // every shot of the problem in one batch
    o.tile = opt ? opt->tile : 0;                  // 0: the default (TMA-staged) variant
    o.shots_per_cta = opt ? opt->shots_per_cta : 0;
    it->P->opt = o;
    FWI_TRY_B(begin_call(it->P, &it->prob.model, &it->prob.geom, pr.wavelet, false, it->c, it->tabC));
    if (it->c.pl.B != pr.geom.nshots)
      return bail(fail(FWI_ERR_BUDGET, "problem " + std::to_string(i) + " does not fit the budget with all its shots"));
    if (i == 0) {
      b->tma = it->c.pl.tma;
      b->shape = it->c.pl.shape;
      if (!b->tma && b->shape != 0)
        return bail(fail(FWI_ERR_UNSUPPORTED, "batches run the TMA variants or shared-memory variant 1"));
    }
    Carve srcC = it->tabC;
    FWI_TRY_B(build_source_table(it->c, 0, pr.geom.nshots, srcC, it->src));
    const size_t fs = (size_t)it->P->L.fstride;
    CUDA_TRY_B(cudaMemsetAsync(it->c.W.U0, 0, fs * pr.geom.nshots * sizeof(float), b->st));
    CUDA_TRY_B(cudaMemsetAsync(it->c.W.U1, 0, fs * pr.geom.nshots * sizeof(float), b->st));
    used += it->c.pl.bytes;
  }
  std::stable_sort(b->items.begin(), b->items.end(),
                   [](const BatchProblem* a, const BatchProblem* c) { return a->prob.nt > c->prob.nt; });
  if (!b->items.empty()) {
    b->w[0] = b->items[0]->P->wx;
    b->w[1] = b->items[0]->P->wy;
    b->uniform_w = true;
    for (const BatchProblem* it : b->items)
      if (std::memcmp(&it->P->wx, &b->w[0], sizeof(AxisW)) != 0 ||
          std::memcmp(&it->P->wy, &b->w[1], sizeof(AxisW)) != 0)
        b->uniform_w = false;
  }
  // descriptors and units (problems longest first: the running ones are a prefix)
  std::vector<MultiDesc> desc(b->items.size());
  std::vector<MultiUnit> units;
  std::vector<int> prefix;
  for (size_t k = 0; k < b->items.size(); ++k) {
    BatchProblem* it = b->items[k];
    Call& c = it->c;
    StepParams p = base_params(c);
    p.B = it->prob.geom.nshots;
    p.inj_off = it->src.off;
    p.inj_loc = it->src.loc;
    p.inj_vidx = it->src.vidx;
    p.inj_w = it->src.w;
    p.vals = it->prob.wavelet;
    p.smp_node = c.smp_node;
    p.smp_w = c.smp_w;
    p.smp_out = c.W.D;
    p.nrec = it->prob.geom.nrec;
    p.S = 1;
    p.flags = it->P->d_flags + 1;
    p.S = c.pl.S;
    desc[k].p = p;
    desc[k].U0 = c.W.U0;
    desc[k].U1 = c.W.U1;
    desc[k].gx = c.T.gx;
    desc[k].nt = it->prob.nt;
    if (b->tma) {
      const CUtensorMap* m0 = find_map(c, c.W.U0);
      const CUtensorMap* m1 = find_map(c, c.W.U1);
      if (!m0 || !m1) return bail(fail(FWI_ERR_INVALID_ARG, "internal: missing tensor maps"));
      desc[k].map0 = *m0;
      desc[k].map1 = *m1;
    }
    // units: one per tile and shot group (TMA kernels loop S shots in a CTA)
    const int groups = b->tma ? (p.B + p.S - 1) / p.S : p.B;
    long long rank = 0;
    for (int gr = 0; gr < groups; ++gr)
      for (int ty = 0; ty < c.T.gy; ++ty)
        for (int tx = 0; tx < c.T.gx; ++tx) units.push_back({(int)k, tx, ty, gr, rank++});
    prefix.push_back((int)units.size());
  }
  b->max_steps = b->items.empty() ? 0 : b->items[0]->prob.nt - 1;
  b->active_units.assign(std::max(b->max_steps, 0), 0);
  for (int n = 0; n < b->max_steps; ++n) {
    int cnt = 0;
    for (size_t k = 0; k < b->items.size(); ++k)
      if (n < b->items[k]->prob.nt - 1) cnt = prefix[k];
    b->active_units[n] = cnt;
  }
  CUDA_TRY_B(cudaMalloc(&b->d_desc, desc.size() * sizeof(MultiDesc)));
  CUDA_TRY_B(cudaMalloc(&b->d_units, std::max<size_t>(units.size(), 1) * sizeof(MultiUnit)));
  CUDA_TRY_B(cudaMemcpy(b->d_desc, desc.data(), desc.size() * sizeof(MultiDesc), cudaMemcpyHostToDevice));
  if (!units.empty())
    CUDA_TRY_B(cudaMemcpy(b->d_units, units.data(), units.size() * sizeof(MultiUnit), cudaMemcpyHostToDevice));
  CUDA_TRY_B(cudaEventCreate(&b->e0));
  CUDA_TRY_B(cudaEventCreate(&b->e1));
  CUDA_TRY_B(cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming));
  CUDA_TRY_B(cudaStreamCreateWithFlags(&b->ws, cudaStreamNonBlocking));
  CUDA_TRY_B(cudaStreamSynchronize(b->st));
  if (b->use_graph) {
    // set the kernels' attributes outside the capture (zero-unit launch), then
    // capture every launch of a run
    {
      cudaError_t e = b->tma ? launch_step2d_tma_multi(b->d_desc, b->d_units, 0, 0, b->R, b->vd,
                                                       b->shape, b->uniform_w ? b->w : nullptr,
                                                       b->ws)
                             : launch_step2d_multi(b->d_desc, b->d_units, 0, 0, b->R, b->vd, b->ws);
      if (e != cudaSuccess) return bail(fail(FWI_ERR_CUDA, cudaGetErrorString(e)));
    }
    CUDA_TRY_B(cudaStreamBeginCapture(b->ws, cudaStreamCaptureModeThreadLocal));
    fwi_status s = batch_enqueue(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->ws, &g);
    if (s != FWI_OK) {
      if (g) cudaGraphDestroy(g);
      return bail(s);
    }
    if (e != cudaSuccess) return bail(fail(FWI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e)));
    b->graph = g;
    CUDA_TRY_B(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  b->stats.problems = (int)b->items.size();
  b->stats.units = (int64_t)units.size();
  *out = b;
  return FWI_OK;
}

fwi_status fwi_batch_run(fwi_batch* b) {
  if (!b) return fail(FWI_ERR_INVALID_ARG, "batch is NULL");
  CUDA_TRY(cudaSetDevice(b->device));
  // the run follows whatever the caller enqueued on its stream (inputs)
  CUDA_TRY(cudaEventRecord(b->ready, b->st));
  CUDA_TRY(cudaStreamWaitEvent(b->ws, b->ready, 0));
  for (BatchProblem* it : b->items) {
    const size_t fs = (size_t)it->P->L.fstride;
    const int ns = it->prob.geom.nshots;
    CUDA_TRY(cudaMemsetAsync(it->c.W.U0, 0, fs * ns * sizeof(float), b->ws));
    CUDA_TRY(cudaMemsetAsync(it->c.W.U1, 0, fs * ns * sizeof(float), b->ws));
    CUDA_TRY(cudaMemsetAsync(it->P->d_flags, 0, sizeof(int) * 4, b->ws));
  }
  CUDA_TRY(cudaEventRecord(b->e0, b->ws));
  if (b->use_graph) {
    CUDA_TRY(cudaGraphLaunch(b->exec, b->ws));
  } else {
    FWI_TRY(batch_enqueue(b));
  }
  CUDA_TRY(cudaEventRecord(b->e1, b->ws));
  CUDA_TRY(cudaStreamSynchronize(b->ws));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, b->e0, b->e1));
  b->stats.run_ms = ms;
  for (BatchProblem* it : b->items) {
    int flags[4];
    CUDA_TRY(cudaMemcpy(flags, it->P->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags[0]) return fail(FWI_ERR_NONFINITE, "non-finite traces in a batched problem");
  }
  return FWI_OK;
}

fwi_status fwi_batch_stats_get(const fwi_batch* b, fwi_batch_stats* out) {
  if (!b || !out) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  *out = b->stats;
  return FWI_OK;
}

void fwi_batch_destroy(fwi_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->st);
  delete b;
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
  P.fixed_memory = true;
  if (cudaDeviceGetAttribute(&P.nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    P.nsm = 152;
  }
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
  Plan all;   // table bound for every shot in one batch, at the tile variant the call will use
  all.B = geom->nshots;
  if (!resolve_tile(&P, P.opt.tile, &all.tile, &all.shape, &all.tma, &all.x2))
    return fail(FWI_ERR_INVALID_ARG, "tile variant out of range");
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
