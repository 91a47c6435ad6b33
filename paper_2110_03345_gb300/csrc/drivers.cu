// Forward and gradient drivers of the C ABI (fwi_forward, fwi_gradient and
// the split fwi_misfit_forward / fwi_misfit_backward).
//
// Forward modelling and the adjoint-state gradient follow Sec. 2.2 (Eqs.
// 5-9) and Sec. 2.4 (Eq. 10) of the Stride paper: per shot, one forward
// propagation storing h^n = k (L u^n + s^n) (or checkpoints of (u^n, u^{n-1})
// every K steps with per-segment recomputation), the L2 residual, and one
// adjoint propagation backwards in time with the imaging condition fused
// into the adjoint step.  Shots run as a batch dimension of every launch.
#include "fwi_plan.cuh"

namespace fwi {

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
                           CUtensorMap* out, bool interior) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  int bx = 0, by = 0;
  if (interior) tma_box2d_interior(shape, &bx, &by);
  else tma_box2d(P->R, shape, &bx, &by);
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

// 4D tensor map over a 2D history buffer of nsteps x nslots padded fields:
// dims (x = sx, y = rows, slot, step), box = one tile without halo.
fwi_status make_tensor_map_hist(const fwi_plan* P, const float* base, int nslots, int nsteps,
                                int shape, CUtensorMap* out) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  int bx = 0, by = 0;
  tma_box2d_interior(shape, &bx, &by);
  const cuuint64_t dims[4] = {(cuuint64_t)P->L.sx, (cuuint64_t)P->L.rows, (cuuint64_t)nslots,
                              (cuuint64_t)nsteps};
  const cuuint64_t strides[3] = {(cuuint64_t)P->L.sx * sizeof(float),
                                 (cuuint64_t)P->L.fstride * sizeof(float),
                                 (cuuint64_t)P->L.fstride * nslots * sizeof(float)};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled (history) failed with code " + std::to_string((int)r));
  return FWI_OK;
}

// 5D tensor map over a 3D history buffer of nsteps x nslots padded fields:
// dims (x, y, z, slot, step), box = box_w x box_h of one plane.
fwi_status make_tensor_map_hist3d(const fwi_plan* P, const float* base, int nslots, int nsteps,
                                  int box_w, int box_h, CUtensorMap* out) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[5] = {(cuuint64_t)P->L.sx, (cuuint64_t)P->L.rows, (cuuint64_t)P->L.planes,
                              (cuuint64_t)nslots, (cuuint64_t)nsteps};
  const cuuint64_t strides[4] = {(cuuint64_t)P->L.sx * sizeof(float),
                                 (cuuint64_t)P->L.sxy * sizeof(float),
                                 (cuuint64_t)P->L.fstride * sizeof(float),
                                 (cuuint64_t)P->L.fstride * nslots * sizeof(float)};
  const cuuint32_t box[5] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1u, 1u, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled (3D history) failed with code " + std::to_string((int)r));
  return FWI_OK;
}

// 4D tensor map over nslots padded 3D fields: dims (x, y, z, slot); box = a
// 48-float-wide (80 for the two-point kernels) x-y tile (16-byte aligned
// start) with its y halo, one plane.
fwi_status make_tensor_map_3d(const fwi_plan* P, const float* base, int nslots, int shape,
                              bool x2, CUtensorMap* out, int box_w, int box_h) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[4] = {(cuuint64_t)P->L.sx, (cuuint64_t)P->L.rows, (cuuint64_t)P->L.planes,
                              (cuuint64_t)nslots};
  const cuuint64_t strides[3] = {(cuuint64_t)P->L.sx * sizeof(float),
                                 (cuuint64_t)P->L.sxy * sizeof(float),
                                 (cuuint64_t)P->L.fstride * sizeof(float)};
  const cuuint32_t box[4] = {box_w > 0 ? (cuuint32_t)box_w : (x2 ? 80u : 48u),
                             box_h > 0 ? (cuuint32_t)box_h : (cuuint32_t)tma_box3d_rows(P->R, shape),
                             1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled (3D) failed with code " + std::to_string((int)r));
  return FWI_OK;
}

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
  p.smp_group = sample_group(c.ncorner);
  p.dt = (float)P->dt;
  p.nb = P->grid.sponge;
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
  if (c.pl.sc.ext() && !c.pl.tma)
    return (long long)c.T.ntiles() * B * (c.P->grid.ndim == 3 ? EXT_TX * EXT_TY3 : EXT_TX2 / 4 * EXT_TY2);
  const int by = (c.P->grid.ndim == 3) ? tile3_variant(c.pl.shape).by
                 : c.pl.tma ? tile2_tma_variant(c.pl.shape).by : tile2_variant(c.pl.shape).by;
  const int ctas_z = (B + c.pl.S - 1) / c.pl.S;
  return (long long)c.T.ntiles() * ctas_z * 32 * by;
}

const CUtensorMap* find_map(const Call& c, const float* base, int kind) {
  for (const auto& m : c.maps)
    if (m.base == base && m.kind == kind) return &m.map;
  return nullptr;
}

fwi_status launch_step(Call& c, const StepParams& p_in, bool adj) {
  fwi_plan* P = c.P;
  StepParams p = p_in;
  if (!adj && p.nrec > 0 && (long long)p.B * p.nrec * p.smp_group > launch_threads(c, p.B)) {
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
    // the two-point variable-density kernels' operand maps (others ignore them)
    const bool ops = c.pl.x2 && c.vd;
    const CUtensorMap* upm = ops ? find_map(c, p.up, 1) : map;
    const CUtensorMap* kfm = ops ? find_map(c, c.W.kf, 1) : map;
    const CUtensorMap* gm = (ops && adj) ? find_map(c, c.W.G, 1) : map;
    if (!upm || !kfm || !gm || (ops && p.image && !c.hmap_ok))
      return fail(FWI_ERR_INVALID_ARG, "internal: no tensor map for the 3D kernels' operands");
    const CUtensorMap* hm = (ops && p.image) ? &c.hmap : map;
    e = c.pl.x2 ? launch_step3d_x2(p, *map, *bxm, *bym, *upm, *kfm, *gm, *hm, P->R, c.vd, adj,
                                   c.pl.shape, P->st)
                : launch_step3d_tma(p, *map, *bxm, *bym, P->R, c.vd, adj, c.pl.shape, P->st);
  } else if (P->grid.ndim == 3) e = launch_step3d(p, P->R, c.vd, adj, c.pl.shape, P->st);
  else if (c.pl.tma) {
    // u^{n-1} (p.up) without halo; the history map only when the adjoint images
    const CUtensorMap* um = find_map(c, p.up, 1);
    if (!um) return fail(FWI_ERR_INVALID_ARG, "internal: no tensor map for u^{n-1}");
    if (adj && p.image && !c.hmap_ok)
      return fail(FWI_ERR_INVALID_ARG, "internal: no tensor map for the history");
    e = launch_step2d_tma(p, *map, *um, (adj && p.image) ? c.hmap : *um, P->R, c.vd, adj,
                          c.pl.shape, P->st);
  }
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

// One time step of an extended scheme (kernels_ext.cu), counted and timed as
// one stencil launch: the fourth-order scheme's two passes (k w, then the
// update from k w; the adjoint's k L^T lambda, then the update with the
// receiver residuals weighted 12 inside the 1/12 bracket), or the single
// pass of the attenuating leapfrog.
// One pass of an extended scheme: the TMA shot-loop kernels (2D, sponge
// boundary; the tensor map of the stencil input p.x) or kernels_ext.cu.
cudaError_t ext_pass(const Call& c, const StepParams& p, bool adj, int mode) {
  const fwi_plan* P = c.P;
  if (c.pl.tma && P->grid.ndim == 3) {
    // the two-point plane ring: p.x's map, b_x / b_y and the operand maps
    const CUtensorMap* xm = find_map(c, p.x);
    if (!xm) return cudaErrorInvalidValue;
    const CUtensorMap* bxm = c.vd ? find_map(c, c.W.bx) : xm;
    const CUtensorMap* bym = c.vd ? find_map(c, c.W.by) : xm;
    const CUtensorMap* upm = c.vd ? find_map(c, p.up, 1) : xm;
    const CUtensorMap* kfm = c.vd ? find_map(c, c.W.kf, 1) : xm;
    const CUtensorMap* gm = (c.vd && adj) ? find_map(c, c.W.G, 1) : xm;
    const bool img = c.vd && adj && p.image;
    if (!bxm || !bym || !upm || !kfm || !gm || (img && !c.hmap_ok)) return cudaErrorInvalidValue;
    return launch_step3d_x2_ext(p, *xm, *bxm, *bym, *upm, *kfm, *gm, img ? c.hmap : *xm, P->R,
                                c.vd, adj, mode, P->st);
  }
  if (c.pl.tma) {
    // p.x with halo, p.up without, and the history fields the adjoint images with
    const CUtensorMap* map = find_map(c, p.x);
    const CUtensorMap* um = find_map(c, p.up, 1);
    const CUtensorMap* ucm = find_map(c, p.u, 1);
    if (!map || !um || !ucm) return cudaErrorInvalidValue;
    const bool img = adj && p.image && mode != EXT_KW;
    if (img && (!c.hmap_ok || (mode == EXT_T4 && !c.h2map_ok))) return cudaErrorInvalidValue;
    return launch_step2d_tma_ext(p, *map, *um, img ? c.hmap : *um,
                                 (img && mode == EXT_T4) ? c.h2map : *um, *ucm, P->R, c.vd, adj,
                                 mode, P->st);
  }
  return launch_ext(p, P->grid.ndim, P->R, c.vd, adj, mode, P->st);
}

fwi_status ext_step(Call& c, const StepParams& p_in, bool adj) {
  fwi_plan* P = c.P;
  StepParams p = p_in;
  const int nd = P->grid.ndim;
  if (!adj && p.nrec > 0 && (long long)p.B * p.nrec * p.smp_group > launch_threads(c, p.B)) {
    cudaError_t e = launch_sample(p, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
    p.nrec = 0;
  }
  const bool prof = P->opt.profile > 0 &&
                    (c.fwd_launches + c.adj_launches) % P->opt.profile == 0;
  p.flags = P->d_flags + 1;
  p.S = c.pl.tma ? c.pl.S : 1;
  p.att = c.W.ATT;
  p.q = adj ? c.W.QA : c.W.QF;
  if (p.inj_scale == 0.f) p.inj_scale = 1.f;
  if (prof) FWI_TRY(record_event(P, adj ? 1 : 0));
  cudaError_t e;
  if (c.pl.sc.t4) {
    StepParams a = p;   // pass 1 (forward) / pass A (adjoint): k (L x + s) into KW
    a.x = p.u;
    a.out = c.W.KW;
    a.hist = nullptr;
    a.hist2 = nullptr;
    a.image = 0;
    if (adj) a.inj_off = nullptr;   // the residuals enter the second pass only
    e = ext_pass(c, a, adj, EXT_KW);
    if (e == cudaSuccess) {
      StepParams b = p;   // pass 2 / B: the update from k w (k L^T lambda)
      b.x = c.W.KW;
      b.nrec = 0;
      if (!adj) b.vals = c.W.D2Q;   // s^{n+1} - 2 s^n + s^{n-1}
      else b.inj_scale = 12.f;      // 12 P^T r inside the 1/12 bracket
      e = ext_pass(c, b, adj, EXT_T4);
    }
    c.launches += 2;
  } else {
    p.x = p.u;
    e = ext_pass(c, p, adj, c.pl.sc.att == 0 ? EXT_ATT0 : EXT_ATT2);
    c.launches++;
  }
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("stencil launch: ") + cudaGetErrorString(e));
  if (prof) {
    FWI_TRY(record_event(P, adj ? 1 : 0));
    if (adj) c.adj_timed++;
    else c.fwd_timed++;
  }
  const int64_t pts = (int64_t)p.B * P->L.nx * P->L.ny * P->L.nz;
  if (adj) { c.adj_launches++; c.adj_points += pts; }
  else { c.fwd_launches++; c.fwd_points += pts; }
  return FWI_OK;
}

// One PML time step (kernels_pml.cu), counted and timed as one stencil
// launch: the u update (u^{n+1} over u^{n-1}, q^{n+1}, h^n), then the phi
// update from u^{n+1} and q^{n+1}.
fwi_status pml_step(Call& c, const StepParams& p_in) {
  fwi_plan* P = c.P;
  StepParams p = p_in;
  const int nd = P->grid.ndim;
  if (p.nrec > 0 && (long long)p.B * p.nrec * p.smp_group > launch_threads(c, p.B)) {
    cudaError_t e = launch_sample(p, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
    p.nrec = 0;
  }
  const bool prof = P->opt.profile > 0 &&
                    (c.fwd_launches + c.adj_launches) % P->opt.profile == 0;
  p.x = p.u;
  p.q = c.W.PQ;
  for (int d = 0; d < 3; ++d) p.ph[d] = c.W.PH[d];
  if (prof) FWI_TRY(record_event(P, 0));
  cudaError_t e = launch_pml(p, nd, P->R, c.vd, PML_U, P->st);
  if (e == cudaSuccess) {
    StepParams b = p;
    b.x = p.up;            // u^{n+1}
    b.nrec = 0;
    b.inj_off = nullptr;
    b.hist = nullptr;
    e = launch_pml(b, nd, P->R, c.vd, PML_PHI, P->st);
  }
  c.launches += 2;
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("PML launch: ") + cudaGetErrorString(e));
  if (prof) {
    FWI_TRY(record_event(P, 0));
    c.fwd_timed++;
  }
  c.fwd_launches++;
  c.fwd_points += (int64_t)p.B * P->L.nx * P->L.ny * P->L.nz;
  return FWI_OK;
}

// Forward sweep of one batch: steps n = n0 .. n1-1 starting from (A = u^{n0},
// Bf = u^{n0-1}).  hist_base: full history [n][B][fs] (n indexed from 0) or a
// segment buffer indexed from n0; sample: record d^n for each step.
fwi_status forward_steps(Call& c, int nb, int shot0, const DevTable& src, float*& A, float*& Bf,
                         int n0, int n1, float* hist_base, int hist_n0, bool sample,
                         int K_ckpt, float* CK, float* hist2_base) {
  fwi_plan* P = c.P;
  const size_t fs = (size_t)P->L.fstride;
  StepParams p = base_params(c);
  p.B = nb;
  p.inj_off = src.off;
  p.inj_loc = src.loc;
  p.inj_vidx = src.vidx;
  p.inj_row = src.row;
  p.inj_crowded = src.crowded || (P->grid.ndim == 3 && c.ncorner > 8);   // 3D: sinc points
  p.inj_w = src.w;
  p.vals = c.wavelet;
  p.smp_node = c.smp_node;
  p.smp_w = c.smp_w;
  p.smp_out = c.D;
  p.nrec = sample ? c.geom->nrec : 0;
  const bool ext = c.pl.sc.ext();
  const bool pml = c.pl.sc.pml;
  const size_t cm = (size_t)c.pl.sc.ckpt_fields();
  for (int n = n0; n < n1; ++n) {
    if (K_ckpt > 0 && n % K_ckpt == 0) {
      // checkpoint j: (u^n, u^{n-1}) and the scheme's other state (the
      // Laplacian of u^{n-1} for y = 2 attenuation; q and phi for the PML)
      const size_t j = n / K_ckpt;
      float* dst = CK + cm * j * fs * c.pl.B;
      CUDA_TRY(cudaMemcpyAsync(dst, A, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
      CUDA_TRY(cudaMemcpyAsync(dst + fs * c.pl.B, Bf, fs * nb * sizeof(float),
                               cudaMemcpyDeviceToDevice, P->st));
      for (size_t i = 0; i < c.fstate.size(); ++i)
        CUDA_TRY(cudaMemcpyAsync(dst + (2 + i) * fs * c.pl.B, c.fstate[i], fs * nb * sizeof(float),
                                 cudaMemcpyDeviceToDevice, P->st));
    }
    p.u = A;
    p.up = Bf;
    p.hist = hist_base ? hist_base + (size_t)(n - hist_n0) * fs * c.pl.B : nullptr;
    p.hist2 = hist2_base ? hist2_base + (size_t)(n - hist_n0) * fs * c.pl.B : nullptr;
    p.step_off = n;
    p.smp_off = (long long)n * c.pl.B * c.geom->nrec;
    if (pml) FWI_TRY(pml_step(c, p));
    else if (ext) FWI_TRY(ext_step(c, p, false));
    else FWI_TRY(launch_step(c, p, false));
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
  // (the fourth-order scheme is stable to sqrt(3) times that)
  const double tf = c.pl.sc.t4 ? std::sqrt(3.0) : 1.0;
  const double lim1 = cfl_limit(1, P->grid.order) * tf;
  const double cfl = (double)vmax * P->dt * std::sqrt(sum);
  if (cfl > 0.95 * lim1) {
    char buf[192];
    std::snprintf(buf, sizeof(buf), "CFL %.4f exceeds 0.95 x the %s limit (%.4f) for vp_max %.1f",
                  cfl / std::sqrt((double)P->grid.ndim), c.pl.sc.t4 ? "fourth-order scheme's" : "leapfrog",
                  0.95 * tf * cfl_limit(P->grid.ndim, P->grid.order), (double)vmax);
    return fail(FWI_ERR_UNSTABLE_CFL, buf);
  }
  if (c.pl.sc.att >= 0) {
    CUDA_TRY(cudaMemsetAsync(c.W.ATT, 0, fs * sizeof(float), P->st));
    CUDA_TRY(cudaMemsetAsync(P->d_stats + 4, 0, 2 * sizeof(unsigned int), P->st));
    e = launch_att_prep(P->L, m->vp, m->param, m->alpha0, c.pl.sc.att, P->dt, c.W.ATT,
                        P->d_stats + 4, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    unsigned int as[2];
    CUDA_TRY(cudaMemcpyAsync(as, P->d_stats + 4, sizeof(as), cudaMemcpyDeviceToHost, P->st));
    CUDA_TRY(cudaStreamSynchronize(P->st));
    if (as[1] != 0) return fail(FWI_ERR_NONFINITE, "alpha0 holds negative or non-finite values");
    if (c.pl.sc.att == 2) {
      // the y = 2 term is explicit: with r = k lambda_max (lambda_max the
      // largest eigenvalue of -lap) and s = r * (2 alpha0 vp / dt) the step is
      // stable for r + 2 s <= 4; checked with the maxima of vp and of the
      // coefficient (conservative) at 0.95^2 of the bound
      float amax;
      std::memcpy(&amax, &as[0], 4);
      const double cl = cfl_limit(1, P->grid.order);
      const double r = (double)vmax * P->dt * (double)vmax * P->dt * sum * 4.0 / (cl * cl);
      if (r * (1.0 + 2.0 * (double)amax) > 4.0 * 0.95 * 0.95) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "the y = 2 attenuation term is unstable at this step: r (1 + 2 max 2 alpha0 vp / dt) "
                      "= %.3f exceeds 0.95^2 x 4 (r = %.3f)", r * (1.0 + 2.0 * (double)amax), r);
        return fail(FWI_ERR_UNSTABLE_CFL, buf);
      }
    }
  }
  if (c.pl.sc.t4) {
    e = launch_second_difference(c.wavelet, c.W.D2Q, (long long)c.geom->nshots * c.geom->nsrc, P->nt,
                                 P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
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
                      const float* wavelet, bool grad, Call& c, Carve& tabC, bool split) {
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
  Scheme sc;
  FWI_TRY(resolve_scheme(P, model, &sc));
  FWI_TRY(choose_plan(P, geom, c.vd, grad, c.pl, split, sc));
  FWI_TRY(ensure_arena(P, c.pl.bytes));
  Carve C(P->arena);
  carve_work(P, c.pl, geom, c.vd, C, c.W);
  if (C.off > P->arena_cap) return fail(FWI_ERR_BUDGET, "workspace carve exceeds allocation");
  c.fstate.clear();
  if (c.W.QF) c.fstate.push_back(c.W.QF);
  if (c.W.PQ) c.fstate.push_back(c.W.PQ);
  for (float* ph : c.W.PH)
    if (ph) c.fstate.push_back(ph);
  if (c.pl.tma) {
    const bool three = P->grid.ndim == 3;
    for (float* buf : {c.W.U0, c.W.U1, c.W.F0, c.W.F1, c.W.KW}) {
      if (!buf) continue;
      Call::MapEnt m{buf, {}};
      if (three) FWI_TRY(make_tensor_map_3d(P, buf, c.pl.B, c.pl.shape, c.pl.x2, &m.map));
      else FWI_TRY(make_tensor_map(P, buf, c.pl.B, c.pl.shape, &m.map));
      c.maps.push_back(m);
      if (!three) {   // the 2D kernels also stage u^{n-1} by TMA
        Call::MapEnt mi{buf, {}, 1};
        FWI_TRY(make_tensor_map(P, buf, c.pl.B, c.pl.shape, &mi.map, true));
        c.maps.push_back(mi);
      }
    }
    if (three && c.vd && c.pl.x2) {
      // the two-point variable-density kernels read u^{n-1} (lambda^{k+1}), k
      // and g by TMA in 64 x BY plane tiles
      const int by = tile3_variant(c.pl.shape).by;
      for (float* buf : {c.W.U0, c.W.U1, c.W.F0, c.W.F1}) {
        if (!buf) continue;
        Call::MapEnt m{buf, {}, 1};
        FWI_TRY(make_tensor_map_3d(P, buf, c.pl.B, c.pl.shape, true, &m.map, 64, by));
        c.maps.push_back(m);
      }
      Call::MapEnt mk{c.W.kf, {}, 1};
      FWI_TRY(make_tensor_map_3d(P, c.W.kf, 1, c.pl.shape, true, &mk.map, 64, by));
      c.maps.push_back(mk);
      if (c.W.G) {   // gradient slots (gradient plans)
        Call::MapEnt mg{c.W.G, {}, 1};
        FWI_TRY(make_tensor_map_3d(P, c.W.G, c.pl.B, c.pl.shape, true, &mg.map, 64, by));
        c.maps.push_back(mg);
      }
    }
    if (three && c.vd) {
      // the two-point kernels stage b_x on the tile rows (80 x BY) and b_y on
      // the tile columns (64 x BY + 2R); the one-point kernels whole planes
      const int by = tile3_variant(c.pl.shape).by;
      const int bw[2] = {c.pl.x2 ? 80 : 0, c.pl.x2 ? 64 : 0};
      const int bh[2] = {c.pl.x2 ? by : 0, c.pl.x2 ? by + 2 * P->R : 0};
      const float* bufs[2] = {c.W.bx, c.W.by};
      for (int i = 0; i < 2; ++i) {
        Call::MapEnt m{bufs[i], {}};
        FWI_TRY(make_tensor_map_3d(P, bufs[i], 1, c.pl.shape, c.pl.x2, &m.map, bw[i], bh[i]));
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
  // the extended schemes' stencil inputs k w (k L^T lambda) are read with
  // their halo: their padding must hold zeros (only the interior is written)
  if (c.W.KW) CUDA_TRY(cudaMemsetAsync(c.W.KW, 0, (size_t)P->L.fstride * c.pl.B * sizeof(float), P->st));
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

void delete_saved(SavedGrad* s) { delete s; }

BatchBufs batch_bufs(const Call& c, int j) {
  const size_t fs = (size_t)c.P->L.fstride;
  const size_t B = (size_t)c.pl.B;
  const size_t k = c.pl.split ? (size_t)j : 0;
  const int nt = c.P->nt;
  BatchBufs b;
  b.D = c.W.D + k * (size_t)nt * B * c.geom->nrec;
  b.CK = c.W.CK ? c.W.CK + k * fs * B * (size_t)c.pl.sc.ckpt_fields() * (size_t)c.pl.nck : nullptr;
  b.H = (c.pl.K == 0) ? c.W.H + k * fs * B * (size_t)std::max(nt - 1, 1) : c.W.H;
  b.H2 = nullptr;
  if (c.W.H2) b.H2 = (c.pl.K == 0) ? c.W.H2 + k * fs * B * (size_t)std::max(nt - 1, 1) : c.W.H2;
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
  for (float* f : c.fstate)   // lap u^{-1} = 0; q^0 = 0, phi^0 = 0
    CUDA_TRY(cudaMemsetAsync(f, 0, fs * nb * sizeof(float), P->st));
  FWI_TRY(forward_steps(c, nb, shot0, src, A, Bf, 0, nt - 1, K == 0 ? bb.H : nullptr, 0, true,
                        K, bb.CK, K == 0 ? bb.H2 : nullptr));
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
  if (c.W.QA) CUDA_TRY(cudaMemsetAsync(c.W.QA, 0, fs * nb * sizeof(float), P->st));
  const bool ext = c.pl.sc.ext();
  const size_t cm = (size_t)c.pl.sc.ckpt_fields();
  StepParams p = base_params(c);
  p.B = nb;
  p.inj_off = c.rec_tab.off;
  p.inj_loc = c.rec_tab.loc;
  p.inj_vidx = c.rec_tab.vidx;
  p.inj_row = c.rec_tab.row;
  p.inj_crowded = c.rec_tab.crowded || (P->grid.ndim == 3 && c.ncorner > 8);
  p.inj_w = c.rec_tab.w;
  p.vals = c.D;
  p.g = c.W.G;
  p.nrec = 0;
  int seg_lo = -1, seg_hi = -1;
  auto hist_at = [&](int n) -> float* {
    if (K == 0) return bb.H + (size_t)n * fs * B;
    return bb.H + (size_t)(n - seg_lo) * fs * B;
  };
  auto hist2_at = [&](int n) -> float* {
    if (!bb.H2) return nullptr;
    if (K == 0) return bb.H2 + (size_t)n * fs * B;
    return bb.H2 + (size_t)(n - seg_lo) * fs * B;
  };
  auto ensure_segment = [&](int n) -> fwi_status {
    if (K == 0 || (n >= seg_lo && n < seg_hi)) return FWI_OK;
    const int js = n / K;
    seg_lo = js * K;
    seg_hi = std::min(seg_lo + K, nt - 1);
    float* FA = c.W.U0;
    float* FB = c.W.U1;
    const float* ck = bb.CK + cm * (size_t)js * fs * B;
    CUDA_TRY(cudaMemcpyAsync(FA, ck, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
    CUDA_TRY(cudaMemcpyAsync(FB, ck + fs * B, fs * nb * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
    for (size_t i = 0; i < c.fstate.size(); ++i)
      CUDA_TRY(cudaMemcpyAsync(c.fstate[i], ck + (2 + i) * fs * B, fs * nb * sizeof(float),
                               cudaMemcpyDeviceToDevice, P->st));
    return forward_steps(c, nb, shot0, src, FA, FB, seg_lo, seg_hi, bb.H, seg_lo, false, 0, nullptr,
                         bb.H2);
  };
  if (c.pl.sc.pml) {
    // PML adjoint (kernels_pml.cu): ubar^{n+1} in XN, ubar^n in XC, c^n, qbar,
    // the phi adjoints; ubar^{nt-1} = P^T r^{nt-1}, ubar^{nt-2} = P^T r^{nt-2}
    float* XN = LA;
    float* XC = LB;
    for (float* f : {c.W.PC, c.W.PQB, c.W.PHB[0], c.W.PHB[1], c.W.PHB[2]})
      if (f) CUDA_TRY(cudaMemsetAsync(f, 0, fs * nb * sizeof(float), P->st));
    const int nd = P->grid.ndim;
    for (int m = 0; m < 2 && nt - 1 - m >= 0; ++m) {
      StepParams pi = p;
      pi.step_off = (long long)(nt - 1 - m) * B * c.geom->nrec;
      cudaError_t e = launch_inject_buckets(pi, m == 0 ? XN : XC, c.T.tx, c.T.ty, c.T.zc, c.T.gx,
                                            c.T.gy, P->st);
      if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
      c.launches++;
    }
    for (int n = nt - 2; n >= 0; --n) {
      FWI_TRY(ensure_segment(n));
      const bool prof = P->opt.profile > 0 &&
                        (c.fwd_launches + c.adj_launches) % P->opt.profile == 0;
      if (prof) FWI_TRY(record_event(P, 1));
      StepParams pa = p;
      pa.up = XN;
      pa.out = c.W.PC;
      pa.q = c.W.PQB;
      for (int d = 0; d < 3; ++d) pa.ph[d] = c.W.PHB[d];
      pa.hist = hist_at(n);
      pa.image = 1;
      pa.step_off = (long long)(n - 1) * B * c.geom->nrec;
      if (n < 1) pa.inj_off = nullptr;   // no residual before the record
      cudaError_t e = launch_pml(pa, nd, P->R, c.vd, PML_A, P->st);
      if (e == cudaSuccess) {
        StepParams pb = p;
        pb.x = c.W.PC;
        pb.up = XC;
        for (int d = 0; d < 3; ++d) pb.ph[d] = c.W.PHB[d];
        pb.inj_off = nullptr;
        e = launch_pml(pb, nd, P->R, c.vd, PML_B, P->st);
      }
      if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("PML launch: ") + cudaGetErrorString(e));
      c.launches += 2;
      if (prof) {
        FWI_TRY(record_event(P, 1));
        c.adj_timed++;
      }
      c.adj_launches++;
      c.adj_points += (int64_t)nb * P->L.nx * P->L.ny * P->L.nz;
      std::swap(XN, XC);
    }
    return FWI_OK;
  }
  // the 2D leapfrog adjoint reads h^k by TMA through a map of this batch's
  // history buffer (nt - 1 steps, or one segment of K)
  c.hmap_ok = c.h2map_ok = false;
  if (c.pl.tma && P->grid.ndim == 3 && c.pl.x2 && c.vd) {
    FWI_TRY(make_tensor_map_hist3d(P, bb.H, B, K == 0 ? std::max(nt - 1, 1) : K, 64,
                                   tile3_variant(c.pl.shape).by, &c.hmap));
    c.hmap_ok = true;
  }
  if (c.pl.tma && P->grid.ndim == 2) {
    const int nsteps = K == 0 ? std::max(nt - 1, 1) : K;
    FWI_TRY(make_tensor_map_hist(P, bb.H, B, nsteps, c.pl.shape, &c.hmap));
    c.hmap_ok = true;
    if (bb.H2) {
      FWI_TRY(make_tensor_map_hist(P, bb.H2, B, nsteps, c.pl.shape, &c.h2map));
      c.h2map_ok = true;
    }
  }
  for (int k = nt - 1; k >= 1; --k) {
    p.image = (k <= nt - 2) ? 1 : 0;
    if (p.image) {
      FWI_TRY(ensure_segment(k));
      p.hist = hist_at(k);
      p.hist2 = hist2_at(k);
      p.hstep = (int)((size_t)(p.hist - bb.H) / (fs * B));
    } else {
      p.hist = nullptr;
      p.hist2 = nullptr;
    }
    p.u = LA;
    p.up = LB;
    p.step_off = (long long)k * B * c.geom->nrec;
    if (ext) FWI_TRY(ext_step(c, p, true));
    else FWI_TRY(launch_step(c, p, true));
    std::swap(LA, LB);
    if (c.Dw) {   // dJ/dq^{k-1}: lambda^{k-1} sampled at the sources (weights / cell volume)
      const int nsrc = c.geom->nsrc;
      cudaError_t e = launch_sample_slots(LA, (long long)fs, c.ws_node, c.ws_w, c.ncorner,
                                          nb * nsrc, nsrc, c.Dw,
                                          (long long)(k - 1) * B * nsrc, P->st);
      if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
      c.launches++;
    }
  }
  if (nt >= 2) {   // imaging term of lambda^0
    FWI_TRY(ensure_segment(0));
    cudaError_t e;
    if (c.pl.sc.t4) {
      // k L^T lambda^0 (the first adjoint pass alone), then the two terms
      StepParams a = p;
      a.x = LA;
      a.u = LA;
      a.out = c.W.KW;
      a.inj_off = nullptr;
      a.hist = nullptr;
      a.hist2 = nullptr;
      a.image = 0;
      a.att = c.W.ATT;
      a.flags = P->d_flags + 1;
      e = launch_ext(a, P->grid.ndim, P->R, c.vd, true, EXT_KW, P->st);
      if (e == cudaSuccess)
        e = launch_image_t4(P->L, LA, c.W.KW, hist_at(0), hist2_at(0), c.W.G, nb, c.pl.S, P->st);
      c.launches += 2;
    } else {
      e = launch_image_only(P->L, LA, hist_at(0), c.W.G, nb, c.pl.S, P->st);
      c.launches++;
    }
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  }
  return FWI_OK;
}

// Sum the gradient slots into grad_m (scaled by 1/dt^2), read the misfit of
// `batches` batches (0: none) and finish the call.
fwi_status gradient_finish(Call& c, int batches, double* misfit, float* grad_m) {
  fwi_plan* P = c.P;
  const int G = (c.pl.B + c.pl.S - 1) / c.pl.S;   // gradient slots in use
  if (grad_m) {
    cudaError_t e = launch_grad_finalize(P->L, c.W.G, G, 1.0 / (P->dt * P->dt), grad_m, P->d_flags, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    c.launches++;
  }
  std::vector<double> J(std::max(batches, 1));
  if (batches > 0)
    CUDA_TRY(cudaMemcpyAsync(J.data(), P->d_J, sizeof(double) * batches, cudaMemcpyDeviceToHost, P->st));
  FWI_TRY(finish_call(c));
  double tot = 0.0;
  for (int i = 0; i < batches; ++i) tot += J[i];
  if (batches > 0) *misfit = tot;
  return FWI_OK;
}

}  // namespace fwi

using namespace fwi;

extern "C" {

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
    for (float* f : c.fstate)
      CUDA_TRY(cudaMemsetAsync(f, 0, fs * nb * sizeof(float), P->st));
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
  if (!grad_m) return fail(FWI_ERR_INVALID_ARG, "grad_m is NULL");
  return fwi_misfit_backward_ex(P, grad_m, nullptr);
}

fwi_status fwi_misfit_backward_ex(fwi_plan* P, float* grad_m, float* grad_wavelet) {
  if (!P) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
  if (!grad_m && !grad_wavelet) return fail(FWI_ERR_INVALID_ARG, "grad_m and grad_wavelet are both NULL");
  SavedGrad* S = P->saved;
  if (!S) return fail(FWI_ERR_INVALID_ARG, "no pending fwi_misfit_forward on this plan");
  if (grad_wavelet && (S->c.pl.sc.t4 || S->c.pl.sc.pml))
    return fail(FWI_ERR_UNSUPPORTED,
                "the wavelet gradient of the fourth-order scheme and of the PML is not implemented");
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
  // dJ/dq workspace: per-step source samples and the batch's sampling table
  const int nsrc = S->geom.nsrc;
  const size_t npt = (size_t)c.pl.B * nsrc;
  void* wbuf = nullptr;
  if (st == FWI_OK && grad_wavelet) {
    const size_t bytes = align_up((size_t)P->nt * npt * 4, 256) + 2 * align_up(npt * c.ncorner * 4, 256);
    e = pool_alloc(&wbuf, bytes, P->st, P->device);
    if (e != cudaSuccess) {
      cudaGetLastError();
      wbuf = nullptr;
      st = fail(FWI_ERR_BUDGET, std::string("dJ/dq workspace: ") + cudaGetErrorString(e));
    } else {
      Carve wc(static_cast<char*>(wbuf));
      c.Dw = wc.take<float>((size_t)P->nt * npt);
      int* node = wc.take<int>(npt * c.ncorner);
      float* w = wc.take<float>(npt * c.ncorner);
      c.ws_node = node;
      c.ws_w = w;
    }
  }
  int batch = 0;
  for (int shot0 = 0; shot0 < S->geom.nshots && st == FWI_OK; shot0 += c.pl.B, ++batch) {
    const int nb = std::min(c.pl.B, S->geom.nshots - shot0);
    Carve srcC = S->tabC;
    DevTable src;
    st = build_source_table(c, shot0, nb, srcC, src);
    if (st == FWI_OK && c.Dw) {
      e = cudaMemsetAsync(c.Dw, 0, (size_t)P->nt * npt * 4, P->st);   // dJ/dq^{nt-1} = 0
      if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
      if (st == FWI_OK)
        st = build_source_sampling(c, shot0, nb, const_cast<int*>(c.ws_node),
                                   const_cast<float*>(c.ws_w));
    }
    if (st == FWI_OK) st = gradient_adjoint_batch(c, batch, shot0, nb, src);
    if (st == FWI_OK && c.Dw) {
      e = launch_traces_out(c.Dw, grad_wavelet, c.pl.B, shot0, nb, nsrc, P->nt, P->d_flags, P->st);
      if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
      c.launches++;
    }
    if (st == FWI_OK && shot0 + c.pl.B < S->geom.nshots) {
      e = cudaStreamSynchronize(P->st);
      if (e != cudaSuccess) st = fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  double J = 0.0;
  if (st == FWI_OK) st = gradient_finish(c, 0, &J, grad_m);
  if (wbuf) {
    cudaStreamSynchronize(P->st);
    cudaFreeAsync(wbuf, P->st);
    cudaGetLastError();
  }
  c.Dw = nullptr;
  c.ws_node = nullptr;
  c.ws_w = nullptr;
  delete_saved(S);
  return st;
}

}  // extern "C"
