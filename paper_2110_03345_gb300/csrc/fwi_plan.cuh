// Internal declarations shared by the host-side translation units of the
// library (plan.cu, tables.cu, drivers.cu, batch.cu, fwi_noalloc.cu): the plan
// object, the per-call workspace plan and the interpolation tables.  Not part
// of the C ABI.
#pragma once
#include "fwi.h"
#include "fwi_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace fwi {

// Records msg as the calling thread's last error (fwi_last_error) and returns s.
fwi_status fail(fwi_status s, const std::string& msg);
void set_last_error(const std::string& msg);

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

// Central-difference weights (standard Taylor weights of the stated order):
// second derivative w2[0..R], first derivative w1[1..R] (antisymmetric).
void fd_weights(int order, double* w2, double* w1);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

struct SavedGrad;
void delete_saved(SavedGrad* s);

}  // namespace fwi

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
  fwi::Layout L{};
  int R = 4;
  double h[3] = {1, 1, 1};  // spacing (x, y, z)
  int n3[3] = {1, 1, 1};    // extents (x, y, z)
  double c_ref = 0.0;
  bool sponge_ready = false;
  fwi::AxisW wx{}, wy{}, wz{};
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
  fwi::SavedGrad* saved = nullptr;  // state kept by fwi_misfit_forward for fwi_misfit_backward
  bool fixed_memory = false;   // buffers supplied by the caller: never allocate
  ~fwi_plan() { fwi::delete_saved(saved); }
};

namespace fwi {

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

// Bi-/tri-linear stencil of one point: nodes (x, y, z) and weights.
struct Corners {
  int n;
  int node[8][3];
  double w[8];
};

// Interpolation stencil of one point for the plan's interp option: n nodes
// (x, y, z at node[3 i .. 3 i + 2]) and their weights.  Bi-/tri-linear: the
// 2^ndim corners; sinc: the (2r)^ndim Kaiser-windowed sinc nodes.
struct PointSt {
  int n = 0;
  std::vector<int> node;
  std::vector<double> w;
};

// Tile geometry of the stencil kernels for entry bucketing.
struct TileGeo {
  int gx, gy, nzc, tx, ty, zc;
  int ntiles() const { return gx * gy * nzc; }
};

struct Entry {
  int bucket;
  int loc;
  int vidx;
  float w;
};

// Host-side bucket tables, laid out [off | loc | vidx | w].
struct HostTable {
  std::vector<int> off, loc, vidx;
  std::vector<float> w;
  std::vector<int> row;   // 2D: per bucket, the first entry of each tile row (rows + 1 values)
  int max_row = 0;        // 2D: most entries in one tile row of one bucket
};

struct DevTable {
  const int* off = nullptr;
  const int* loc = nullptr;
  const int* vidx = nullptr;
  const float* w = nullptr;
  const int* row = nullptr;
  int crowded = 0;        // some tile row holds more than 32 entries
};

// Time scheme and attenuation of a call: the leapfrog of the default
// kernels, or an extended scheme run by the kernels of kernels_ext.cu.
struct Scheme {
  bool t4 = false;   // fourth order in time (options.time_order == 4)
  int att = -1;      // attenuation power y (0 or 2), -1 for none
  bool pml = false;  // perfectly matched layer instead of the sponge (options.boundary == 1)
  int ndim = 2;
  bool ext() const { return t4 || att >= 0 || pml; }
  // PML state besides u^n, u^{n-1}: q (3D) and one phi per axis
  int pml_state() const { return pml ? ndim + (ndim == 3 ? 1 : 0) : 0; }
  int hist_fields() const { return t4 ? 2 : 1; }         // stored per step (F and k w)
  int ckpt_fields() const {                               // u^n, u^{n-1} and the other state
    return 2 + (att == 2 ? 1 : 0) + pml_state();
  }
  int fwd_slot_fields() const { return (t4 ? 1 : 0) + (att == 2 ? 1 : 0) + pml_state(); }
  // adjoint: lap state (y = 2); c, qbar (3D) and the phi adjoints (PML)
  int adj_slot_fields() const { return (att == 2 ? 1 : 0) + (pml ? 1 + pml_state() : 0); }
  int model_fields() const { return att >= 0 ? 1 : 0; }  // attenuation coefficient
};

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
  Scheme sc;            // extended scheme (then tma, x2 = false, S = 1, tile = 0)
};

// Per-call device state carved out of the arena.
struct Work {
  float *kf = nullptr, *lnr = nullptr, *bx = nullptr, *by = nullptr, *bz = nullptr;
  float *U0 = nullptr, *U1 = nullptr, *F0 = nullptr, *F1 = nullptr, *G = nullptr;
  float *H = nullptr, *CK = nullptr, *D = nullptr;
  // extended schemes: attenuation coefficient, k w scratch, Laplacian states
  // (forward, adjoint), second history field, second time difference of the wavelets
  float *ATT = nullptr, *KW = nullptr, *QF = nullptr, *QA = nullptr, *H2 = nullptr, *D2Q = nullptr;
  // PML: q and phi (forward), c, qbar and the phi adjoints (adjoint)
  float *PQ = nullptr, *PC = nullptr, *PQB = nullptr;
  float *PH[3] = {nullptr, nullptr, nullptr}, *PHB[3] = {nullptr, nullptr, nullptr};
  double* partials = nullptr;
  int npartials = 0;
};

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
    int kind = 0;   // 0: tile with halo; 1: 2D tile without halo (u^{n-1})
  };
  std::vector<MapEnt> maps;   // TMA descriptors of the wavefield buffers
  CUtensorMap hmap{};         // 2D TMA adjoint: the current batch's history buffer
  CUtensorMap h2map{};        // and its second history field (fourth-order scheme)
  bool hmap_ok = false, h2map_ok = false;
  std::vector<float*> fstate; // forward state besides u^n, u^{n-1} (checkpointed with them)
  int64_t launches = 0;
  int64_t fwd_launches = 0, adj_launches = 0;
  int64_t fwd_points = 0, adj_points = 0;
  int64_t fwd_timed = 0, adj_timed = 0;   // launches that carried events
  // optional dJ/dq (the adjoint of wavelet -> traces sampled at the sources):
  // per-step samples [nt][B][nsrc] and the batch's source sampling table
  float* Dw = nullptr;
  const int* ws_node = nullptr;   // [B * nsrc][ncorner] node of each source corner
  const float* ws_w = nullptr;    // its weight / cell volume
};

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

// Pointers of batch j's kept state: traces/residuals, checkpoints, history.
struct BatchBufs {
  float* D;
  float* CK;
  float* H;
  float* H2;   // fourth-order scheme: second history field
};

// ---- plan.cu: plan memory, layout, validation, workspace planning
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t st, int device);
size_t device_available(int device);
fwi_status ensure_arena(fwi_plan* P, size_t bytes);
fwi_status ensure_tab(fwi_plan* P, size_t bytes);
double cfl_limit(int ndim, int order);
long long padded_field_floats(const fwi_grid* g);
fwi_status validate_grid(const fwi_grid* g);
void build_layout(fwi_plan* P);
fwi_status build_sponge(fwi_plan* P);
fwi_status validate_geometry(const fwi_plan* P, const fwi_geometry* g);
bool resolve_tile(const fwi_plan* P, int t, int* id, int* shape, bool* tma, bool* x2 = nullptr);
size_t field_bytes(const fwi_plan* P);
size_t model_bytes(const fwi_plan* P, bool vd, const Scheme& sc);
size_t slot_bytes(const fwi_plan* P, const fwi_geometry* g, bool grad, int K, const Scheme& sc);
size_t persist_bytes_per_shot(const fwi_plan* P, const fwi_geometry* g, int K, const Scheme& sc);
size_t split_slot_bytes(const fwi_plan* P, int K, const Scheme& sc);
size_t fixed_bytes(const fwi_plan* P, const fwi_geometry* g, bool vd, int B, const Scheme& sc);
// The scheme of a call from the plan's options and the model (NULL: none).
fwi_status resolve_scheme(const fwi_plan* P, const fwi_model* m, Scheme* sc);
fwi_status choose_plan(const fwi_plan* P, const fwi_geometry* g, bool vd, bool grad, Plan& out,
                       bool split = false, const Scheme& sc = Scheme());
void carve_work(fwi_plan* P, const Plan& pl, const fwi_geometry* g, bool vd, Carve& C, Work& W);

// ---- tables.cu: interpolation and injection tables
Corners point_corners(const fwi_plan* P, const double* xyz);
// Nodes per point for an interp option and dimension (4 / 8 linear, 64 / 512 sinc).
int interp_nodes(int interp, int ndim);
// Per-axis Kaiser-windowed sinc weights of a point at x grid units on an axis
// of n nodes: first node and the 2 r weights; false if the point lies closer
// than r - 1 nodes to a face.
bool sinc_axis(double x, long long n, int* first, double* w);
bool point_stencil(const fwi_plan* P, const double* xyz, PointSt& out);
long long node_index(const Layout& L, const int* n);
TileGeo tile_geo(const fwi_plan* P, int tile, bool tma, bool x2 = false, bool ext = false);
void add_entry(std::vector<Entry>& E, const TileGeo& T, int slot, const int* node, int vidx,
               float w);
// Entries grouped by bucket and sorted by tile-local index; with rows > 0 (2D
// tiles of rows x tx points) also the per-row entry ranges of every bucket.
HostTable bucket(const std::vector<Entry>& E_in, int nbuckets, int rows = 0, int tx = 0);
size_t table_bytes(const HostTable& H);
fwi_status upload_table(fwi_plan* P, const HostTable& H, Carve& C, DevTable& D);
fwi_status build_source_table(Call& c, int shot0, int nb, Carve& C, DevTable& D);
fwi_status prepare_common(Call& c, Carve& tabC);
size_t tables_bound(const fwi_plan* P, const fwi_geometry* g, const Plan& pl);

// ---- fwi_noalloc.cu
fwi_status check_on_device(const void* ptr, const char* name, int dev);

// ---- drivers.cu: launches, forward and adjoint sweeps, call set-up
// 2D tensor maps over nslots padded fields: the tile with halo (interior =
// false) or without (interior = true); make_tensor_map_hist: a history
// buffer of nsteps x nslots fields, box = one tile without halo
fwi_status make_tensor_map_hist(const fwi_plan* P, const float* base, int nslots, int nsteps,
                                int shape, CUtensorMap* out);
// a 3D history buffer of nsteps x nslots fields: (x, y, z, slot, step), box
// box_w x box_h x 1 x 1 x 1
fwi_status make_tensor_map_hist3d(const fwi_plan* P, const float* base, int nslots, int nsteps,
                                  int box_w, int box_h, CUtensorMap* out);
fwi_status make_tensor_map(const fwi_plan* P, const float* base, int nslots, int shape,
                           CUtensorMap* out, bool interior = false);
// box_w / box_h > 0 override the box's x extent and rows
fwi_status make_tensor_map_3d(const fwi_plan* P, const float* base, int nslots, int shape,
                              bool x2, CUtensorMap* out, int box_w = 0, int box_h = 0);
fwi_status record_event(fwi_plan* P, int kind);
StepParams base_params(Call& c);
long long launch_threads(const Call& c, int B);
const CUtensorMap* find_map(const Call& c, const float* base, int kind = 0);
fwi_status launch_step(Call& c, const StepParams& p_in, bool adj);
fwi_status forward_steps(Call& c, int nb, int shot0, const DevTable& src, float*& A, float*& Bf,
                         int n0, int n1, float* hist_base, int hist_n0, bool sample,
                         int K_ckpt, float* CK, float* hist2_base = nullptr);
fwi_status ext_step(Call& c, const StepParams& p_in, bool adj);
fwi_status pml_step(Call& c, const StepParams& p_in);
fwi_status final_sample(Call& c, int nb, const float* A, int n);
fwi_status prepare_model(Call& c);
fwi_status begin_call(fwi_plan* P, const fwi_model* model, const fwi_geometry* geom,
                      const float* wavelet, bool grad, Call& c, Carve& tabC, bool split = false);
fwi_status finish_call(Call& c);
BatchBufs batch_bufs(const Call& c, int j);
fwi_status gradient_forward_batch(Call& c, int j, int shot0, int nb, const DevTable& src,
                                  const float* observed, float* traces_opt);
fwi_status gradient_adjoint_batch(Call& c, int j, int shot0, int nb, const DevTable& src);
fwi_status gradient_finish(Call& c, int batches, double* misfit, float* grad_m);
fwi_status build_source_sampling(Call& c, int shot0, int nb, int* d_node, float* d_w);

}  // namespace fwi
