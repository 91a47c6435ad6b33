// Internal declarations of the GB300 acoustic FWI library (not part of the ABI).
//
// Device data layout (one "field" = one FP32 array over the padded grid):
//   x (last axis) is padded by OX = 8 floats on the left and rounded up to a
//   multiple of 128 plus 8 on the right, so every row starts 32-byte aligned
//   and float4 loads of a tile plus its halo never leave the allocation;
//   y and z are padded by the stencil radius R on both sides and rounded up
//   to a multiple of 64 (the largest tile height).  The padding holds zeros,
//   which is the u = 0 boundary condition behind the sponge, so stencil
//   loads need no bounds checks.  Per-shot fields are stacked [B][fstride].
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fwi {

constexpr int OX = 8;          // x padding (floats) before the interior
constexpr int TILE_X = 128;    // tile width of the 2D kernels (32 threads x float4)
constexpr int ROUND_Y = 64;    // y (and z) extents are rounded to this
constexpr int MAX_SLOT_TILES = 1 << 20;

struct Layout {
  int ndim;
  int nx, ny, nz;        // interior extents (nz = 1 in 2D)
  int R;                 // stencil radius
  int ox, oy, oz;        // interior origin in padded coordinates
  int sx;                // row stride (floats)
  int rows;              // padded rows (y)
  int planes;            // padded planes (z; 1 in 2D)
  long long sxy;         // plane stride (floats)
  long long fstride;     // floats per field
  int nx_r, ny_r, nz_r;  // rounded interior extents covered by tiles
  __host__ __device__ long long index(int z, int y, int x) const {
    return (long long)(z + oz) * sxy + (long long)(y + oy) * sx + (x + ox);
  }
};

// Scaled stencil weights for one axis: w2[j] / h^2 and w1[j] / h.
struct AxisW {
  float w2[6];
  float w1[6];
};

// Parameters of one stencil launch (forward or adjoint step).
struct StepParams {
  const float* u;      // u^n (adjoint: lambda^k), [B][fstride]
  float* up;           // in: u^{n-1} (lambda^{k+1}); out: u^{n+1} (lambda^{k-1})
  const float* kf;     // k = (vp dt)^2, [fstride]
  const float* bx;     // density gradient d(ln rho)/dx etc. (variable density)
  const float* by;
  const float* bz;
  const float* spx;    // sponge a_d(i) = sigma_d(i) dt / 2, per axis, rounded length
  const float* spy;
  const float* spz;
  float* hist;         // forward: store k(L u + s) here (or null); adjoint: read h^k
  float* g;            // adjoint imaging accumulator [B][fstride] (or null)
  long long fstride;
  long long sxy;
  int sx;
  int nx, ny, nz;
  int ox, oy, oz;
  AxisW wx, wy, wz;
  float ih2[3];          // 1 / h_d^2 and 1 / h_d (x, y, z): scales of the unscaled
  float ih1[3];          // compile-time weights of the 3D TMA kernels
  // sparse injection, bucketed by (slot, tile): entries e in [off[s*T+t], off[s*T+t+1]),
  // ordered by inj_loc within a bucket (stable: same-node entries keep their order)
  const int* inj_off;
  const int* inj_loc;    // tile-local linear index (2D: ly*TX+lx; 3D: (lz*TY+ly)*TX+lx)
  const int* inj_vidx;   // index into vals (before step_off)
  const int* inj_row;    // 2D: per bucket, entry range of each tile row (TY + 1 values)
  int inj_crowded;       // some tile row (2D) holds more than 32 entries; 3D: sinc points
  int hstep;             // 2D TMA adjoint: step of hist within the history buffer's tensor map
  const float* inj_w;    // weight (source: w/dV; receiver residual: w)
  const float* vals;
  long long step_off;
  int ntiles;            // tiles per slot
  // receiver sampling of u (forward only): out[smp_off + b*nrec + r]
  const int* smp_node;   // [nrec][ncorner] padded index within a shot field
  const float* smp_w;
  float* smp_out;
  long long smp_off;
  int nrec;
  int ncorner;
  int smp_group;         // lanes per (slot, receiver) sample: 1, or 32 for sinc points
  int B;                 // shot slots in this launch
  int image;             // adjoint: accumulate g -= lambda^k h^k
  int zchunk;            // 3D: planes per CTA
  int nzc;               // 3D: z chunks
  int S;                 // shots per CTA (TMA kernels); gradient slot of shot s is s / S
  int* flags;            // device error flags (bit 1: a bounded wait timed out)
  // extended schemes (kernels_ext.cu, kernels2d_tma_ext.cu): stencil input, per-point
  // attenuation coefficient, Laplacian state and a second history field
  const float* x;        // field whose stencil is taken (u^n, k w^n, lambda^k or k y^k)
  float* out;            // pass 1 / A of the fourth-order scheme: k (L x + s)
  const float* att;      // y = 0: alpha0 vp dt; y = 2: 2 alpha0 vp / dt
  float* q;              // y = 2: Laplacian of the previous step (updated in place)
  float* hist2;          // fourth-order scheme: k w^n (forward store, adjoint read)
  float inj_scale;       // factor on injected values (fourth-order adjoint pass B: 12)
  // perfectly matched layer (kernels_pml.cu): auxiliary fields phi_x, phi_y,
  // phi_z (forward) or their adjoints, the time step, the layer width
  float* ph[3];
  float dt;
  int nb;
};

// Lanes per receiver sample: the 64- / 512-node sinc points split their
// nodes over a warp (one thread each would serialise 64-512 gathers in the
// few threads that sample and hold up their CTAs), the 4 / 8 corners of the
// linear points take one thread.
inline int sample_group(int ncorner) { return ncorner > 8 ? 32 : 1; }

#ifdef __CUDACC__
// First injection entry of each plane lz = 0 .. nplanes of a 3D bucket whose
// entries sort by tile-local index ((lz * TY + y) * TX + x): pe[lz] (one
// bisection per plane by the CTA's threads; visible after a barrier).
__device__ __forceinline__ void plane_entries(const StepParams& p, int bucket, int nplanes,
                                              int plane_pts, int tid, int nthreads, int* pe) {
  const int e0 = p.inj_off[bucket], e1 = p.inj_off[bucket + 1];
  for (int k = tid; k <= nplanes; k += nthreads) {
    const int lim = k * plane_pts;
    int lo = e0, hi = e1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(p.inj_loc + mid) < lim) lo = mid + 1;
      else hi = mid;
    }
    pe[k] = lo;
  }
}

// Receiver sampling d = P u^n by a launch's first threads: thread gid serves
// the sample (slot, receiver) = gid / G with the nodes c = gid % G + k G,
// and a group of G > 1 lanes (a whole warp, gid aligned to it) sums its
// partial sums by shuffles in a fixed order.  Every thread of a warp calls it.
__device__ __forceinline__ void sample_receivers(const StepParams& p, long long gid) {
  const int G = p.smp_group > 1 ? p.smp_group : 1;
  if (p.nrec <= 0 || gid >= (long long)p.B * p.nrec * G) return;
  const long long pt = gid / G;
  const int lane = (int)(gid - pt * G);
  const int bb = (int)(pt / p.nrec);
  const int r = (int)(pt - (long long)bb * p.nrec);
  const float* ub = p.u + (long long)bb * p.fstride;
  const int* nd = p.smp_node + (long long)r * p.ncorner;
  const float* w = p.smp_w + (long long)r * p.ncorner;
  float acc = 0.f;
  for (int c = lane; c < p.ncorner; c += G) acc = fmaf(w[c], ub[nd[c]], acc);
  if (G > 1) {
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane != 0) return;
  }
  p.smp_out[p.smp_off + pt] = acc;
}
#endif

// Extended schemes (kernels_ext.cu): shared-memory staged tiles of 128 x 16
// points, a float4 per thread (2D), or 32 x 8 columns streamed along z, one
// point per thread (3D).
enum ExtMode {
  EXT_KW = 0,    // out = k (L x + s)                  (4th order, first pass)
  EXT_T4 = 1,    // F = x + k (L x + s) / 12, update     (4th order, second pass)
  EXT_ATT0 = 2,  // leapfrog with per-point damping alpha0 vp dt   (y = 0)
  EXT_ATT2 = 3,  // leapfrog with the Laplacian-difference term     (y = 2)
};
constexpr int EXT_TX2 = 128, EXT_TX = 32, EXT_TY2 = 16, EXT_TY3 = 8, EXT_ZC = 32;
// Perfectly matched layer passes (kernels_pml.cu), same tiles as the extended
// schemes: forward u update, forward phi update, adjoint pass A (the phi and
// q adjoints into ubar^{n+1}, c^n, imaging), adjoint pass B (L^T(k c) and the
// phi adjoints).
enum PmlMode { PML_U = 0, PML_PHI = 1, PML_A = 2, PML_B = 3 };
cudaError_t launch_pml(const StepParams& p, int ndim, int R, bool vd, int mode, cudaStream_t st);
// field[slot][node] += w vals[vidx + step_off] over the buckets of p.B slots
// (tile geometry tx x ty x zc, gx x gy tiles per plane chunk)
cudaError_t launch_inject_buckets(const StepParams& p, float* field, int tx, int ty, int zc, int gx,
                                  int gy, cudaStream_t st);
cudaError_t launch_ext(const StepParams& p, int ndim, int R, bool vd, bool adj, int mode,
                       cudaStream_t st);
// out[i] = q[i+1] - 2 q[i] + q[i-1] along the last axis of rows x nt samples
// (q = 0 outside the record): the source's second time difference
cudaError_t launch_second_difference(const float* q, float* out, long long rows, int nt,
                                     cudaStream_t st);
// g[b / S] -= lam[b] F[b] + ky[b] kw[b] / 12 for the nb slots of a batch
// (S shots share a gradient slot)
cudaError_t launch_image_t4(const Layout& L, const float* lam, const float* ky, const float* F,
                            const float* kw, float* g, int nb, int S, cudaStream_t st);
// attenuation coefficient field from vp (param 0) or m (param 1) and alpha0:
// y = 0: alpha0 vp dt; y = 2: 2 alpha0 vp / dt (zero in the padding);
// stats[0] |= bits of its maximum, stats[1] += count of bad alpha0 values
cudaError_t launch_att_prep(const Layout& L, const float* vp, int param, const float* alpha0,
                            int y, double dt, float* att, unsigned int* stats, cudaStream_t st);

// Multi-problem forward step (kernels2d.cu): one launch advances every unit
// (problem, tile, shot slot) of the table by one time step.  The descriptor
// holds the problem's StepParams except the per-step fields, which the kernel
// derives from the global step n and the two wavefield buffers.
struct MultiDesc {
  CUtensorMap map0;   // TMA descriptors of U0 and U1 (TMA-staged kernels)
  CUtensorMap map1;
  CUtensorMap imap0;  // and of their tiles without halo (u^{n-1} staged by TMA)
  CUtensorMap imap1;
  StepParams p;
  float* U0;   // u^n for even n (then u^{n-1} for odd n), [B][fstride]
  float* U1;
  int gx;      // tiles along x
  int nt;      // time samples of the problem (active while n < nt - 1)
};
struct MultiUnit {
  int prob, tx, ty, slot;
  long long rank;  // CTA rank among the problem's units (receiver sampling)
};

// Tile variants of the 2D kernels: rows per thread x thread rows.
struct Tile2 { int ry, by; };
constexpr int NUM_TILE2 = 4;
__host__ __device__ inline Tile2 tile2_variant(int v) {
  switch (v) {
    case 1: return {2, 16};
    case 2: return {4, 4};
    case 3: return {2, 8};
    default: return {4, 8};
  }
}
// Tile shapes of the TMA-staged 2D kernels (one or two rows per thread keep
// registers at <= 64 so that 32-64 warps per SM hide the memory latency).
__host__ __device__ inline Tile2 tile2_tma_variant(int v) {
  switch (v) {
    case 1: return {1, 16};
    case 2: return {2, 16};
    case 3: return {2, 8};
    default: return {1, 32};
  }
}
// 3D tile variants: thread rows (tile 32 x by) and z chunk (at most MAX_ZCHUNK)
constexpr int MAX_ZCHUNK = 64;
struct Tile3 { int by, zc; };
constexpr int NUM_TILE3 = 4;
__host__ __device__ inline Tile3 tile3_variant(int v) {
  switch (v) {
    case 1: return {8, 64};
    case 2: return {16, 32};
    case 3: return {8, 32};
    default: return {8, 16};   // short chunks: more CTAs per shot against the wave tail
  }
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_step2d(const StepParams& p, int R, bool vd, bool adj, int tile,
                          cudaStream_t st);
cudaError_t launch_step3d(const StepParams& p, int R, bool vd, bool adj, int tile,
                          cudaStream_t st);
size_t step2d_smem(int R, bool vd, bool adj, int tile);
// Multi-problem forward step, TMA-staged (kernels2d_tma_multi.cu); units are
// (problem, tile, shot group) with the tile shape tile2_tma_variant(tile).
// w: {x, y} stencil weights shared by every problem, or null when they differ.
cudaError_t launch_step2d_tma_multi(const MultiDesc* descs, const MultiUnit* units, int nunits,
                                    int n, int R, bool vd, int tile, const AxisW* w,
                                    cudaStream_t st);
// Multi-problem forward step over `nunits` units (128 x 32 tiles, one shot per CTA).
cudaError_t launch_step2d_multi(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                                int R, bool vd, cudaStream_t st);
// TMA-staged 2D kernels with a loop over p.S shots per CTA (kernels2d_tma.cu);
// tile = 0..NUM_TILE2-1 selects the same tile shapes as tile2_variant.
// um maps p.up without halo (box tma_box2d_interior); hm maps the adjoint's
// history buffer as (x, y, slot, step) with the same box, step p.hstep (read
// only when p.image); both move u^{n-1} and h^k by TMA with the tile.
cudaError_t launch_step2d_tma(const StepParams& p, const CUtensorMap& map, const CUtensorMap& um,
                              const CUtensorMap& hm, int R, bool vd, bool adj, int tile,
                              cudaStream_t st);
void tma_box2d(int R, int tile, int* bx, int* by);
void tma_box2d_interior(int tile, int* bx, int* by);
// The extended schemes' 2D kernels on the same pipeline (kernels2d_tma_ext.cu):
// mode = EXT_KW / EXT_T4 / EXT_ATT0 / EXT_ATT2, map = the tensor map of the
// stencil input p.x for tile shape 1 (128 x 16), um of p.up without halo, hm
// / h2m of the history fields (read by the adjoint when p.image), ucm of
// p.u without halo (read by the fourth-order update), p.S shots per CTA.
cudaError_t launch_step2d_tma_ext(const StepParams& p, const CUtensorMap& map,
                                  const CUtensorMap& um, const CUtensorMap& hm,
                                  const CUtensorMap& h2m, const CUtensorMap& ucm, int R, bool vd,
                                  bool adj, int mode, cudaStream_t st);
size_t step3d_smem(int R, bool vd, bool adj, int tile);
// TMA-staged 3D kernels (kernels3d_tma.cu): um maps the wavefield buffer p.u
// as (x, y, z, slot); bxm / bym map the b_x / b_y fields (variable-density
// adjoint only).  tile = 0..NUM_TILE3-1 as tile3_variant.
cudaError_t launch_step3d_tma(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                              const CUtensorMap& bym, int R, bool vd, bool adj, int tile,
                              cudaStream_t st);
int tma_box3d_rows(int R, int tile);
// Two-point TMA-staged 3D kernels (kernels3d_x2.cu): 64 x BY columns, the
// same tensor maps with an 80-float-wide box; bit-identical to the above.
// The variable-density kernels also read per-plane operands by TMA: upm
// (p.up) and kfm (k, one slot), in the adjoint also gm (the gradient slots),
// map (x, y, z, slot) with a 64 x BY box, hm the history buffer as (x, y, z,
// slot, step), step p.hstep (read when p.image); other launches ignore them.
cudaError_t launch_step3d_x2(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                             const CUtensorMap& bym, const CUtensorMap& upm,
                             const CUtensorMap& kfm, const CUtensorMap& gm,
                             const CUtensorMap& hm, int R, bool vd, bool adj, int tile,
                             cudaStream_t st);
// The extended schemes on the same kernels (kernels3d_x2_ext.cu; tile
// variant 12: 64 x 8 columns): mode = EXT_KW / EXT_T4 / EXT_ATT0, xm the map
// of the stencil input p.x, the other maps as above.
cudaError_t launch_step3d_x2_ext(const StepParams& p, const CUtensorMap& xm, const CUtensorMap& bxm,
                                 const CUtensorMap& bym, const CUtensorMap& upm,
                                 const CUtensorMap& kfm, const CUtensorMap& gm,
                                 const CUtensorMap& hm, int R, bool vd, bool adj, int mode,
                                 cudaStream_t st);

// Auxiliary kernels (aux_kernels.cu)
cudaError_t launch_model_prep(const Layout& L, const float* vp, const float* rho, double dt,
                              int param, float* kf, float* lnr, unsigned int* stats,
                              cudaStream_t st);
cudaError_t launch_density_grad(const Layout& L, const float* lnr, const AxisW& wx,
                                const AxisW& wy, const AxisW& wz, float* bx, float* by,
                                float* bz, cudaStream_t st);
cudaError_t launch_sample(const StepParams& p, cudaStream_t st);
// out[off + pt] = sum_c w[pt][c] u[pt / per_slot][node[pt][c]] for pt < npts: samples of
// per-slot point sets (e.g. the sources of each shot of a batch), nc corners each
cudaError_t launch_sample_slots(const float* u, long long fstride, const int* node, const float* w,
                                int nc, int npts, int per_slot, float* out, long long off,
                                cudaStream_t st);
cudaError_t launch_misfit(const float* d_ws, const float* obs, float* traces_out, int B,
                          int shot0, int nshots_batch, int nrec, int nt, double* partials,
                          int* nonfinite, int npartials, cudaStream_t st);
int misfit_blocks(int nshots_batch, int nrec, int nt);
cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t st);
cudaError_t launch_traces_out(const float* d_ws, float* traces_out, int B, int shot0,
                              int nshots_batch, int nrec, int nt, int* nonfinite,
                              cudaStream_t st);
// g[b / S] -= lam[b] * hist[b] for the nb shot slots of a batch
cudaError_t launch_image_only(const Layout& L, const float* lam, const float* hist, float* g,
                              int nb, int S, cudaStream_t st);
// grad_out = (sum of the G gradient slots) * inv_dt2 on the interior
cudaError_t launch_grad_finalize(const Layout& L, const float* g, int G, double inv_dt2,
                                 float* grad_out, int* nonfinite, cudaStream_t st);

}  // namespace fwi
