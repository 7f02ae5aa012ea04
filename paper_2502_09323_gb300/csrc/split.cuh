// Split solve (included by solve.cu after the engine): one system's
// mixed-precision PCG (Sec. 4's CG with the FP64 iterative refinement of this
// library) on R z-slabs, "ranks", each with its own copy of its planes.
//
// Rank r owns the global interior planes [k0_r, k1_r) (contiguous, sizes
// within one plane of each other) and holds them with one halo plane on
// each side: local plane 0 is global plane k0_r - 1, local plane nzl - 1 is
// global plane k1_r.  Every kernel of the single solve runs unchanged on a
// slab (its work items cover the local planes 1 .. nzl - 2); what a split
// adds is the exchange step:
//   * before the direction kernels, the halo planes of z (written by the
//     last update kernels) are copied from the neighbours' boundary planes
//     into each receiver's own memory (cudaMemcpyPeerAsync: a peer copy when
//     the ranks live on different GPUs); p_old's halos are the p halos
//     exchanged before the last update kernels;
//   * before the update kernels, the halo planes of the new p;
//   * before every FP64 true residual, the halo planes of phi;
//   * after each kernel round, the ranks' partial dot products are added in
//     rank order (one thread, FP64) and the CG update (alpha, or beta, the
//     stopping test, the iteration count) is written to every rank's state,
//     so every rank takes the same decision.  The FP64 residual norms are
//     added in rank order on the host.
// The global boundary planes are Dirichlet planes: the first rank's low halo
// and the last rank's high halo hold zeros (vectors) and the boundary values
// (phi) and are never exchanged.
//
// One rank (R = 1) takes exactly the single solve's arithmetic: its result
// is bit-identical to pb_solve's with the same z-chunk.  With R > 1 only the
// order of the dot-product sums changes.

namespace {

struct Slab {
    int k0 = 0, k1 = 0, nzl = 0;  // owned global planes [k0, k1), local planes
    PadGeo pg{};
    GridGeo gg{};
    double *W[3] = {nullptr, nullptr, nullptr}, *diag = nullptr, *rhs = nullptr, *phi = nullptr;
    uint8_t *code = nullptr;
    float *w32[3] = {nullptr, nullptr, nullptr};
    float *z = nullptr, *pbuf[2] = {nullptr, nullptr}, *d = nullptr;
    CgState *st = nullptr;
    double *partials = nullptr;
    int npartials = 0;
    unsigned int *queue = nullptr;
    float *tpart = nullptr;
    tma::SysEntry host{};
    tma::SysEntry *dev = nullptr;
};

// the rank-ordered sum of the ranks' partials and the CG update, written to
// every rank's state (mode 0: after the direction kernels, 1: after the
// update kernels)
__global__ void k_split_combine(CgState *const *sts, int R, int mode) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    CgState *s0 = sts[0];
    if (s0->done) return;
    double t0 = 0.0, t1 = 0.0;
    int abort = 0;
    for (int r = 0; r < R; ++r) {
        t0 += sts[r]->part0;
        t1 += sts[r]->part1;
        abort |= sts[r]->status == 3;
    }
    CgState n = *s0;
    if (mode == 0) {
        n.sigma = t0;
        if (abort) {
            n.done = 1;
            n.status = 3;
        } else if (n.profile) {
            n.alpha = isfinite(t0) && t0 != 0.0 ? n.rho / t0 : 0.0;
        } else if (!(t0 > 0.0) || !isfinite(t0)) {
            n.done = 1;
            n.status = 1;
        } else {
            n.alpha = n.rho / t0;
        }
    } else {
        n.beta = t0 / n.rho;
        n.rho = t0;
        n.rr = t1;
        n.iter += 1;
        n.cur ^= 1;
        if (abort) {
            n.done = 1;
            n.status = 3;
        } else if (n.profile) {
        } else if (!isfinite(t1)) {
            n.done = 1;
            n.status = 1;
        } else if (t1 <= n.rr_stop) {
            n.done = 1;
            n.status = 0;
        } else if (n.iter >= n.max_iter) {
            n.done = 1;
            n.status = 2;
        }
    }
    for (int r = 0; r < R; ++r) {
        CgState *s = sts[r];
        const unsigned int counter = s->counter;
        *s = n;
        s->counter = counter;
    }
    __threadfence();
}

void slab_free(Slab &sl, cudaStream_t s) {
    void *ptrs[] = {sl.W[0], sl.W[1], sl.W[2], sl.diag, sl.rhs, sl.phi, sl.code, sl.w32[0],
                    sl.w32[1], sl.w32[2], sl.z, sl.pbuf[0], sl.pbuf[1], sl.d, sl.st,
                    sl.partials, sl.queue, sl.tpart, sl.dev};
    for (void *p : ptrs) dfree(p, s);
    sl = Slab();
}

// copy planes [g0, g0 + n) of a global array (plane size ps elements of esz
// bytes) into a slab array from its plane 0
pb_status copy_planes(void *dst, const void *src, long long g0, long long n, long long ps, size_t esz,
                      cudaStream_t s) {
    PB_CUDA_TRY(cudaMemcpyAsync(dst, (const char *)src + (size_t)(g0 * ps) * esz,
                                (size_t)(n * ps) * esz, cudaMemcpyDeviceToDevice, s));
    return PB_OK;
}

pb_status slab_build(const pb_system *sys, Slab &sl, int k0, int k1, int KC, int tw, int dev,
                     cudaStream_t s) {
    const GridGeo &G = sys->g->geo;
    const PadGeo &P = sys->pad;
    sl.k0 = k0;
    sl.k1 = k1;
    sl.nzl = k1 - k0 + 2;
    sl.gg = G;
    sl.gg.nz = sl.nzl;
    sl.gg.N = (long long)G.nx * G.ny * sl.nzl;
    sl.pg = P;
    sl.pg.nz = sl.nzl;
    sl.pg.Np = P.sxy * sl.nzl;
    sl.pg.N = sl.gg.N;
    const long long cN = sl.gg.N, pN = sl.pg.Np, cps = (long long)G.nx * G.ny, pps = P.sxy;
    for (int d = 0; d < 3; ++d) {
        sl.W[d] = (double *)dalloc(8 * cN, s);
        sl.w32[d] = (float *)dalloc(4 * pN, s);
    }
    sl.diag = (double *)dalloc(8 * cN, s);
    sl.rhs = (double *)dalloc(8 * cN, s);
    sl.phi = (double *)dalloc(8 * cN, s);
    sl.code = (uint8_t *)dalloc(pN, s);
    sl.z = (float *)dalloc(4 * pN, s);
    sl.pbuf[0] = (float *)dalloc(4 * pN, s);
    sl.pbuf[1] = (float *)dalloc(4 * pN, s);
    sl.d = (float *)dalloc(4 * pN, s);
    sl.st = (CgState *)dalloc(sizeof(CgState), s);
    sl.npartials = (int)(2 * cdiv(cN, 256) + 64);
    sl.partials = (double *)dalloc(8 * (size_t)sl.npartials, s);
    sl.queue = (unsigned int *)dalloc(4 * sizeof(unsigned int), s);
    const int nitems = tma_items(sl.pg, KC, tw);
    sl.tpart = (float *)dalloc(sizeof(float) * 3 * (size_t)nitems, s);
    sl.dev = (tma::SysEntry *)dalloc(sizeof(tma::SysEntry), s);
    if (!sl.W[0] || !sl.W[1] || !sl.W[2] || !sl.w32[0] || !sl.w32[1] || !sl.w32[2] || !sl.diag ||
        !sl.rhs || !sl.phi || !sl.code || !sl.z || !sl.pbuf[0] || !sl.pbuf[1] || !sl.d || !sl.st ||
        !sl.partials || !sl.queue || !sl.tpart || !sl.dev)
        return PB_ERR_OOM;
    pb_status rc = PB_OK;
    const long long g0 = k0 - 1, n = sl.nzl;
    for (int d = 0; d < 3 && rc == PB_OK; ++d) {
        rc = copy_planes(sl.W[d], sys->W[d], g0, n, cps, 8, s);
        if (rc == PB_OK) rc = copy_planes(sl.w32[d], sys->w32[d], g0, n, pps, 4, s);
    }
    if (rc == PB_OK) rc = copy_planes(sl.diag, sys->diag, g0, n, cps, 8, s);
    if (rc == PB_OK) rc = copy_planes(sl.rhs, sys->rhs, g0, n, cps, 8, s);
    if (rc == PB_OK) rc = copy_planes(sl.phi, sys->bc, g0, n, cps, 8, s);  // phi_0 = boundary values
    if (rc == PB_OK) rc = copy_planes(sl.code, sys->code, g0, n, pps, 1, s);
    if (rc != PB_OK) return rc;
    for (float *q : {sl.z, sl.pbuf[0], sl.pbuf[1], sl.d})
        PB_CUDA_TRY(cudaMemsetAsync(q, 0, 4 * pN, s));
    PB_CUDA_TRY(cudaMemsetAsync(sl.st, 0, sizeof(CgState), s));
    PB_CUDA_TRY(cudaMemsetAsync(sl.queue, 0, 4 * sizeof(unsigned int), s));
    // the slab's launch-table entry (the single solve's, on the slab's buffers)
    tma::SysEntry &e = sl.host;
    for (int c = 0; c < 2 && rc == PB_OK; ++c) {
        pb_system view{};
        view.pad = sl.pg;
        view.code = sl.code;
        rc = tma_maps(&view, MODE_P, sl.z, sl.pbuf[c], nullptr, nullptr, &e.P[c], tw);
        if (rc == PB_OK)
            rc = tma_maps(&view, MODE_U, sl.pbuf[c ^ 1], nullptr, sl.d, sl.z, &e.U[c], tw);
    }
    if (rc != PB_OK) return rc;
    e.pg = sl.pg;
    e.cp = make_c32(sys);
    e.cp.wx = sl.w32[0];
    e.cp.wy = sl.w32[1];
    e.cp.wz = sl.w32[2];
    e.pbuf[0] = sl.pbuf[0];
    e.pbuf[1] = sl.pbuf[1];
    e.x = sl.d;
    e.z = sl.z;
    e.y = nullptr;
    e.st = sl.st;
    e.partials = sl.tpart;
    e.cnt = nullptr;
    tma_entry_geometry(e, sl.pg, KC, tw);
    PB_CUDA_TRY(cudaMemcpyAsync(sl.dev, &e, sizeof(e), cudaMemcpyHostToDevice, s));
    (void)dev;
    return PB_OK;
}

// the two halo planes of a slab vector from its neighbours' boundary planes
// (element size esz, plane size ps elements), into the receiver's memory
pb_status exchange(std::vector<Slab> &sl, int which, long long ps, size_t esz, int dev,
                   cudaStream_t s) {
    const int R = (int)sl.size();
    auto ptr = [&](Slab &x) -> char * {
        switch (which) {
            case 0: return (char *)x.z;
            case 1: return (char *)x.pbuf[0];
            case 2: return (char *)x.pbuf[1];
            default: return (char *)x.phi;
        }
    };
    const size_t bytes = (size_t)ps * esz;
    for (int r = 0; r < R; ++r) {
        char *base = ptr(sl[r]);
        if (r > 0) {  // low halo <- the lower rank's last owned plane
            const char *src = ptr(sl[r - 1]) + (size_t)(sl[r - 1].nzl - 2) * bytes;
            PB_CUDA_TRY(cudaMemcpyPeerAsync(base, dev, src, dev, bytes, s));
        }
        if (r + 1 < R) {  // high halo <- the upper rank's first owned plane
            const char *src = ptr(sl[r + 1]) + bytes;
            PB_CUDA_TRY(cudaMemcpyPeerAsync(base + (size_t)(sl[r].nzl - 1) * bytes, dev, src, dev,
                                            bytes, s));
        }
    }
    return PB_OK;
}

pb_status slab_states(std::vector<Slab> &sl, double rho, double rr0, double rr_stop, int max_iter,
                      pb_system *sys, cudaStream_t s) {
    CgState h{};
    h.rho = rho;
    h.rr0 = rr0;
    h.rr = rr0;
    h.rr_stop = rr_stop;
    h.max_iter = max_iter;
    h.split = 1;
    CgState *stage = sys->h_st + 2;
    *stage = h;
    for (Slab &x : sl)
        PB_CUDA_TRY(cudaMemcpyAsync(x.st, stage, sizeof(CgState), cudaMemcpyHostToDevice, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return PB_OK;
}

// FP64 true residual of every slab (phi halos exchanged first); the norms
// added in rank order on the host
pb_status slab_residual(std::vector<Slab> &sl, pb_system *sys, int dev, cudaStream_t s,
                        double *res2, double *rz) {
    const GridGeo &G = sys->g->geo;
    pb_status rc = exchange(sl, 3, (long long)G.nx * G.ny, 8, dev, s);
    if (rc != PB_OK) return rc;
    static const long long res32 = resident_blocks(k_residual<float>);
    for (Slab &x : sl) {
        unsigned blocks = (unsigned)std::min<long long>(
            std::min<long long>(cdiv(x.gg.N, 256), res32), (long long)x.npartials / 2 - 32);
        k_residual<float><<<blocks, 256, 0, s>>>(x.phi, x.rhs, x.W[0], x.W[1], x.W[2], x.diag,
                                                 x.gg, x.pg, x.z, x.st, x.partials, nullptr,
                                                 x.k0 - 1, G.nz);
        PB_LAUNCH_CHECK();
    }
    // the z halos are refreshed before the first direction kernels
    double a = 0.0, b = 0.0;
    for (Slab &x : sl) {
        PB_CUDA_TRY(cudaMemcpyAsync(sys->h_st + 3, x.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        a += sys->h_st[3].res64;
        b += sys->h_st[3].rz64;
    }
    *res2 = a;
    *rz = b;
    return PB_OK;
}

}  // namespace

pb_status solve_split(pb_system *sys, int R, const pb_solve_opts *o, cudaStream_t s,
                      pb_solve_stats *stats) {
    const double t_start = now_s();
    const double deadline = o->time_budget_s > 0.0 ? t_start + o->time_budget_s : 0.0;
    const GridGeo &G = sys->g->geo;
    const int nint = G.nz - 2;
    if (R < 1 || R > nint || R > 64) {
        set_error("pb_solve_split: ranks must be between 1 and min(64, nz - 2)");
        return PB_ERR_ARG;
    }
    int dev = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    pb_status rc = ensure_solver_ws(sys, PB_MIXED, s);
    if (rc != PB_OK) return rc;
    if ((rc = build_tma_state(sys)) != PB_OK) return rc;
    Tuning tune;
    if ((rc = autotune(sys, PB_MIXED, s, &tune)) != PB_OK) return rc;
    const int KC = std::max(tune.kc, 4), TW = tune.tw;
    const int max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    const int max_outer = o->max_outer > 0 ? o->max_outer : 30;
    const double rtol = o->rtol > 0.0 ? o->rtol : 1e-8;
    const double inner_rtol = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-6;

    std::vector<Slab> sl(R);
    CgState **dsts = nullptr;
    int status = PB_OK, iters = 0, outer = 0;
    double fn2 = 0.0, res2 = 0.0, rz = 0.0;
    do {
        // contiguous slabs of owned planes, sizes within one plane
        for (int r = 0; r < R && rc == PB_OK; ++r) {
            const int k0 = 1 + (int)((long long)nint * r / R);
            const int k1 = 1 + (int)((long long)nint * (r + 1) / R);
            rc = slab_build(sys, sl[r], k0, k1, KC, TW, dev, s);
        }
        if (rc != PB_OK) break;
        dsts = (CgState **)dalloc(sizeof(CgState *) * R, s);
        if (!dsts) {
            rc = PB_ERR_OOM;
            break;
        }
        std::vector<CgState *> hs(R);
        for (int r = 0; r < R; ++r) hs[r] = sl[r].st;
        if (cudaMemcpyAsync(dsts, hs.data(), sizeof(CgState *) * R, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = PB_ERR_CUDA;
            break;
        }
        if ((rc = slab_residual(sl, sys, dev, s, &fn2, &rz)) != PB_OK) break;
        res2 = fn2;
        outer = 1;
        int stagnant = 0;
        const dim3 grid = tma_grid(sys->pad, KC);
        while (fn2 > 0.0 && res2 > rtol * rtol * fn2) {
            if (outer > max_outer || iters >= max_iter) {
                status = PB_ERR_NOCONV;
                break;
            }
            const double rel = sqrt(res2 / fn2);
            double itol = std::max(inner_rtol, 0.5 * rtol / rel);
            if (itol > 0.5) itol = 0.5;
            if ((rc = slab_states(sl, rz, res2, itol * itol * res2, max_iter - iters, sys, s)) != PB_OK)
                break;
            for (Slab &x : sl) {
                cudaMemsetAsync(x.d, 0, 4 * (size_t)x.pg.Np, s);
                cudaMemsetAsync(x.pbuf[0], 0, 4 * (size_t)x.pg.Np, s);
            }
            // inner PCG: chunks of iterations, the host polls rank 0's state
            int cur = 0;
            bool done = false;
            while (!done && rc == PB_OK) {
                for (int c = 0; c < 16 && rc == PB_OK; ++c) {
                    rc = exchange(sl, 0, sys->pad.sxy, 4, dev, s);
                    for (Slab &x : sl)
                        tma_launch<MODE_P>(x.dev, 1, x.host.nitems, x.queue, grid, s, &x.host);
                    k_split_combine<<<1, 32, 0, s>>>(dsts, R, 0);
                    if (rc == PB_OK) rc = exchange(sl, 1 + (cur ^ 1), sys->pad.sxy, 4, dev, s);
                    for (Slab &x : sl)
                        tma_launch<MODE_U>(x.dev, 1, x.host.nitems, x.queue, grid, s, &x.host);
                    k_split_combine<<<1, 32, 0, s>>>(dsts, R, 1);
                    note_launch(2 * R + 2);
                    cur ^= 1;
                }
                if (rc != PB_OK) break;
                if (cudaGetLastError() != cudaSuccess ||
                    cudaMemcpyAsync(sys->h_st, sl[0].st, sizeof(CgState), cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    rc = PB_ERR_CUDA;
                    break;
                }
                done = sys->h_st[0].done;
                // cur is the device's parity: the host issued an iteration
                // after the state was done only as launches that return at once
                cur = sys->h_st[0].cur;
                if (!done && deadline > 0.0 && now_s() > deadline) {
                    status = PB_ERR_TIMEOUT;
                    break;
                }
            }
            if (rc != PB_OK || status == PB_ERR_TIMEOUT) break;
            if (sys->h_st[0].status == 3) {
                set_error("a device-side wait reached its limit in the FP32 PCG kernels");
                status = PB_ERR_TIMEOUT;
                break;
            }
            iters += sys->h_st[0].iter;
            for (Slab &x : sl) {
                k_promote<float><<<cdiv(x.gg.N, 256), 256, 0, s>>>(x.phi, x.d, x.gg, x.pg);
                PB_LAUNCH_CHECK();
            }
            const double prev = res2;
            if ((rc = slab_residual(sl, sys, dev, s, &res2, &rz)) != PB_OK) break;
            ++outer;
            if (res2 > 0.25 * prev) {
                if (++stagnant >= 3) {
                    status = PB_ERR_NOCONV;
                    break;
                }
            } else {
                stagnant = 0;
            }
        }
        if (rc != PB_OK) break;
        // phi of the system: boundary values, then the owned planes
        const long long cps = (long long)G.nx * G.ny;
        if (cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * (size_t)G.N, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            rc = PB_ERR_CUDA;
        for (Slab &x : sl)
            if (cudaMemcpyAsync(sys->phi + (size_t)(x.k0 * cps), x.phi + (size_t)cps,
                                (size_t)((x.k1 - x.k0) * cps) * 8, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                rc = PB_ERR_CUDA;
    } while (false);
    cudaStreamSynchronize(s);
    for (Slab &x : sl) slab_free(x, s);
    dfree(dsts, s);
    cudaStreamSynchronize(s);
    if (rc != PB_OK) return rc;
    sys->fnorm2 = fn2;
    sys->solved = 1;
    if (stats) {
        stats->status = status;
        stats->iters_inner = iters;
        stats->iters_outer = outer;
        stats->kc = KC + 1000 + 10000 * TW;
        stats->true_rel_res = fn2 > 0.0 ? sqrt(res2 / fn2) : 0.0;
        stats->seconds = now_s() - t_start;
        stats->dof = (long long)(G.nx - 2) * (G.ny - 2) * (G.nz - 2);
        stats->model_bytes = (long long)iters * stats->dof * (8 * 4 + 2) + (long long)outer * G.N * 64;
    }
    return (pb_status)status;
}
