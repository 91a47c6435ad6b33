// Plans of the C ABI: creation, options, memory, grid layout, sponge,
// validation of grids and geometries, and the workspace plan of a call
// (batch size, history or checkpoints, kernel variant).  The discretisation
// follows Sec. 2.4 of the Stride paper (Eq. 10; sponge absorbing layer).
#include "fwi_plan.cuh"

namespace fwi {

namespace {
thread_local std::string g_err;
}  // namespace

fwi_status fail(fwi_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

void set_last_error(const std::string& msg) { g_err = msg; }

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

// Resolve fwi_options.tile: 0 selects the default variant.
bool resolve_tile(const fwi_plan* P, int t, int* id, int* shape, bool* tma, bool* x2) {
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

size_t model_bytes(const fwi_plan* P, bool vd, const Scheme& sc) {
  const size_t f = align_up(field_bytes(P), 256);
  return f * (1 + (vd ? 1 + P->grid.ndim : 0) + sc.model_fields());
}

size_t slot_bytes(const fwi_plan* P, const fwi_geometry* g, bool grad, int K, const Scheme& sc) {
  const size_t f = align_up(field_bytes(P), 256);
  const size_t traces = align_up((size_t)P->nt * g->nrec * sizeof(float), 256);
  size_t b = (2 + sc.fwd_slot_fields()) * f + traces;
  if (!grad) return b;
  b += (1 + sc.adj_slot_fields()) * f;  // g slot (and the adjoint Laplacian state)
  const int nt = P->nt;
  const size_t hf = sc.hist_fields();
  if (K == 0) {
    b += (size_t)std::max(nt - 1, 1) * hf * f;
  } else {
    const int nck = (nt - 2) / K + 1;
    b += 2 * f + (size_t)sc.ckpt_fields() * nck * f + (size_t)K * hf * f;
  }
  return b;
}

// Split gradient: bytes kept per shot between the two calls (checkpoints or
// history, and the residual traces), and the per-slot working set.
size_t persist_bytes_per_shot(const fwi_plan* P, const fwi_geometry* g, int K, const Scheme& sc) {
  const size_t f = align_up(field_bytes(P), 256);
  const size_t traces = (size_t)P->nt * g->nrec * sizeof(float);
  if (K == 0) return (size_t)std::max(P->nt - 1, 1) * sc.hist_fields() * f + traces;
  const int nck = (P->nt - 2) / K + 1;
  return (size_t)sc.ckpt_fields() * nck * f + traces;
}

size_t split_slot_bytes(const fwi_plan* P, int K, const Scheme& sc) {
  const size_t f = align_up(field_bytes(P), 256);
  return (5 + sc.fwd_slot_fields() + sc.adj_slot_fields()) * f +
         (K ? (size_t)K * sc.hist_fields() * f : 0) + 4096;
}

size_t fixed_bytes(const fwi_plan* P, const fwi_geometry* g, bool vd, int B, const Scheme& sc) {
  const size_t misfit = align_up((size_t)misfit_blocks(B, g->nrec, P->nt) * 8, 256);
  const size_t d2q = sc.t4 ? align_up((size_t)g->nshots * g->nsrc * P->nt * 4, 256) : 0;
  return model_bytes(P, vd, sc) + misfit + d2q + (4u << 20);
}

fwi_status resolve_scheme(const fwi_plan* P, const fwi_model* m, Scheme* sc) {
  *sc = Scheme();
  const int to = P->opt.time_order;
  if (to != 0 && to != 2 && to != 4)
    return fail(FWI_ERR_INVALID_ARG, "time_order must be 0, 2 or 4");
  sc->t4 = to == 4;
  sc->ndim = P->grid.ndim;
  if (P->opt.boundary != 0 && P->opt.boundary != 1)
    return fail(FWI_ERR_INVALID_ARG, "boundary must be 0 (sponge) or 1 (PML)");
  sc->pml = P->opt.boundary == 1;
  if (m && m->alpha0) {
    if (m->att_power != 0 && m->att_power != 2)
      return fail(FWI_ERR_INVALID_ARG, "att_power must be 0 or 2");
    sc->att = m->att_power;
  }
  if (sc->t4 && sc->att >= 0)
    return fail(FWI_ERR_UNSUPPORTED, "attenuation with the fourth-order time scheme is not implemented");
  if (sc->pml && (sc->t4 || sc->att >= 0))
    return fail(FWI_ERR_UNSUPPORTED, "the PML runs with the second-order scheme without attenuation");
  if (sc->t4 && P->opt.interp != FWI_INTERP_LINEAR)
    return fail(FWI_ERR_UNSUPPORTED, "sinc points with the fourth-order time scheme are not implemented");
  return FWI_OK;
}

fwi_status choose_plan(const fwi_plan* P, const fwi_geometry* g, bool vd, bool grad, Plan& out,
                       bool split, const Scheme& sc) {
  const int ns = g->nshots;
  const size_t budget = P->budget;
  const int K_auto = std::max(2, (int)std::ceil(std::sqrt(2.0 * std::max(P->nt, 2))));
  const long long N = (long long)P->L.nx * P->L.ny * P->L.nz;
  const int B_fill = (int)std::max(1LL, (8LL << 20) / std::max(N, 1LL));  // slots that fill the GPU
  auto fit = [&](int K) {
    size_t fixed = fixed_bytes(P, g, vd, ns, sc);
    size_t per = slot_bytes(P, g, grad, K, sc);
    if (split) {
      // nbatches * B <= ns + B - 1 shots of kept state
      const size_t keep = persist_bytes_per_shot(P, g, K, sc);
      fixed += (size_t)ns * keep;
      per = split_slot_bytes(P, K, sc) + keep;
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
  out.sc = sc;
  if (sc.ext()) {
    // the extended schemes have one tile shape: in 2D (sponge boundary) the
    // TMA shot-loop kernels of 128 x 16 tiles (variant 6), otherwise one
    // shot per CTA (kernels_ext.cu, kernels_pml.cu)
    // in 3D the two-point plane-ring kernels take the fourth-order scheme and
    // the y = 0 term (variant 12); y = 2 and the PML keep kernels_ext.cu /
    // kernels_pml.cu
    const bool tma2 = P->grid.ndim == 2 && !sc.pml;
    const bool x2 = P->grid.ndim == 3 && !sc.pml && (sc.t4 || sc.att == 0);
    out.tile = tma2 ? 6 : (x2 ? 12 : 0);
    out.shape = tma2 ? 1 : (x2 ? 3 : 0);
    out.tma = tma2 || x2;
    out.x2 = x2;
  }
  // slots x z chunks go on grid.z, which CUDA limits to 65535 blocks
  B = std::min(B, std::max(1, 65535 / std::max(1, tile_geo(P, out.shape, out.tma, out.x2,
                                                           sc.ext() && !out.tma).nzc)));
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
  out.bytes = fixed_bytes(P, g, vd, B, sc) + (size_t)B * slot_bytes(P, g, grad, K, sc);
  if (split)
    out.bytes = fixed_bytes(P, g, vd, B, sc) + (size_t)B * split_slot_bytes(P, K, sc) +
                (size_t)out.nbatches * B * persist_bytes_per_shot(P, g, K, sc) + (4u << 20);
  return FWI_OK;
}

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
  const Scheme& sc = pl.sc;
  if (sc.att >= 0) W.ATT = C.take<float>(fs);
  if (sc.t4) W.D2Q = C.take<float>((size_t)g->nshots * g->nsrc * P->nt);
  W.npartials = misfit_blocks(B, g->nrec, P->nt);
  W.partials = C.take<double>(W.npartials);
  W.U0 = C.take<float>(fs * B);
  W.U1 = C.take<float>(fs * B);
  if (sc.t4) W.KW = C.take<float>(fs * B);
  if (sc.att == 2) W.QF = C.take<float>(fs * B);
  if (sc.pml) {
    if (P->grid.ndim == 3) W.PQ = C.take<float>(fs * B);
    for (int d = 0; d < P->grid.ndim; ++d) W.PH[d] = C.take<float>(fs * B);
  }
  const size_t nbk = pl.split ? (size_t)pl.nbatches : 1;   // batches whose state is kept
  W.D = C.take<float>((size_t)P->nt * B * g->nrec * nbk);
  if (pl.gradient) {
    W.G = C.take<float>(fs * B);
    if (sc.att == 2) W.QA = C.take<float>(fs * B);
    if (sc.pml) {
      W.PC = C.take<float>(fs * B);
      if (P->grid.ndim == 3) W.PQB = C.take<float>(fs * B);
      for (int d = 0; d < P->grid.ndim; ++d) W.PHB[d] = C.take<float>(fs * B);
    }
    if (pl.K == 0) {
      W.H = C.take<float>(fs * B * (size_t)std::max(P->nt - 1, 1) * nbk);
      if (sc.t4) W.H2 = C.take<float>(fs * B * (size_t)std::max(P->nt - 1, 1) * nbk);
    } else {
      W.F0 = C.take<float>(fs * B);
      W.F1 = C.take<float>(fs * B);
      W.CK = C.take<float>(fs * B * (size_t)sc.ckpt_fields() * (size_t)pl.nck * nbk);
      W.H = C.take<float>(fs * B * (size_t)pl.K);
      if (sc.t4) W.H2 = C.take<float>(fs * B * (size_t)pl.K);
    }
  }
}

}  // namespace fwi

using namespace fwi;

extern "C" {

const char* fwi_last_error(void) { return fwi::g_err.c_str(); }

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
  if (opt->time_order != 0 && opt->time_order != 2 && opt->time_order != 4)
    return fail(FWI_ERR_INVALID_ARG, "time_order must be 0, 2 or 4");
  if (opt->interp != FWI_INTERP_LINEAR && opt->interp != FWI_INTERP_SINC)
    return fail(FWI_ERR_INVALID_ARG, "interp must be FWI_INTERP_LINEAR or FWI_INTERP_SINC");
  if (opt->boundary != 0 && opt->boundary != 1)
    return fail(FWI_ERR_INVALID_ARG, "boundary must be 0 (sponge) or 1 (PML)");
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
  Scheme sc;
  FWI_TRY(resolve_scheme(plan, nullptr, &sc));
  FWI_TRY(choose_plan(plan, geom, true, gradient != 0, pl, false, sc));
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

}  // extern "C"
