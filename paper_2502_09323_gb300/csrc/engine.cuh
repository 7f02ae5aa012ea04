// Continuous-batching solve engine (included by solve.cu).
//
// A pump thread owns one CUDA stream and keeps a fixed-capacity launch table
// of mixed-precision solves resident on the device.  Every replay of one
// captured graph runs `chunk` FP32 PCG iterations (direction + update
// kernels) of every system in the table; a system that is submitted while
// others are running takes a free slot and joins at the next replay, and a
// finished one leaves its slot at once.  The FP64 iterative refinement of
// the CG solve of Eq. matrixequation (Sec. 3.1; CG as in Sec. 4) runs per
// system between its inner solves: the host sees an
// inner solve end in the state mirror copied back after every replay and
// queues that system's promotion, true residual and refinement step, whose
// decision (next inner tolerance, convergence, stagnation, iteration limits)
// is taken on the device by k_ir_step with the same arithmetic as the
// single-system solver, so the host never waits for a refinement step.
//
// A system's arithmetic depends only on the system and its z-chunk, not on
// the other systems in the table or on when it joined: its reductions are
// finalised per system in a fixed order, and its iteration count is decided
// by its own device state.

namespace {

// FP64 iterative-refinement controller of one slot (device side)
struct IrCtl {
    double fn2;         // |f - A phi_0|^2: the reference for the relative residual
    double res2;        // latest true residual norm^2
    double rtol, inner_rtol;
    long long ticket;   // the occupant this record belongs to
    int max_iter, max_outer;
    int iters, outer, stagnant;
    int final_;         // 1 once the solve has ended
    int status;         // pb_status of the ended solve
    int gen;            // refinement steps taken (the host waits for the next)
};

struct EngineSlot {
    CgState st;
    IrCtl ctl;
};

// One refinement decision for one slot.  first = 1 right after the initial
// residual; otherwise after an inner solve, its promotion and the new true
// residual.  Arms the next inner solve in the slot's CG state, or ends the
// solve (done = 1 keeps the PCG kernels off the slot).
__global__ void k_ir_step(EngineSlot *slot, int first, long long ticket, double rtol,
                          double inner_rtol, int max_iter, int max_outer) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    CgState &st = slot->st;
    IrCtl &c = slot->ctl;
    if (first) {
        c.ticket = ticket;
        c.rtol = rtol;
        c.inner_rtol = inner_rtol;
        c.max_iter = max_iter;
        c.max_outer = max_outer;
        c.fn2 = st.res64;
        c.res2 = c.fn2;
        c.iters = 0;
        c.outer = 1;
        c.stagnant = 0;
        c.final_ = 0;
        c.status = PB_OK;
        c.gen = 0;
    } else if (st.status == 3) {
        // a device-side wait of the PCG kernels reached its limit
        c.final_ = 1;
        c.status = PB_ERR_TIMEOUT;
    } else {
        c.iters += st.iter;
        const double prev = c.res2;
        c.res2 = st.res64;
        c.outer += 1;
        if (c.res2 > 0.25 * prev) {
            if (++c.stagnant >= 3) {
                c.final_ = 1;
                c.status = PB_ERR_NOCONV;
            }
        } else {
            c.stagnant = 0;
        }
    }
    if (!c.final_) {
        if (!(c.fn2 > 0.0 && c.res2 > c.rtol * c.rtol * c.fn2)) {
            c.final_ = 1;
            c.status = PB_OK;
        } else if (c.outer > c.max_outer || c.iters >= c.max_iter) {
            c.final_ = 1;
            c.status = PB_ERR_NOCONV;
        }
    }
    if (c.final_) {
        st.done = 1;
    } else {
        const double rel = sqrt(c.res2 / c.fn2);
        double itol = fmax(c.inner_rtol, 0.5 * c.rtol / rel);
        if (itol > 0.5) itol = 0.5;
        const double rz = st.rz64, res64 = st.res64;
        CgState h{};
        h.rho = rz;
        h.rr0 = c.res2;
        h.rr = c.res2;
        h.rr_stop = itol * itol * c.res2;
        h.max_iter = c.max_iter - c.iters;
        h.res64 = res64;
        h.rz64 = rz;
        st = h;
    }
    c.gen += 1;
    __threadfence();
}

struct EngineJob {
    pb_system *sys = nullptr;
    long long ticket = 0;
    cudaEvent_t ready = nullptr;  // recorded on the submitting stream
    int kc = 8;
    int tw = tma::TWDEF;          // tile width of the TMA-staged kernels
    bool oct = false;             // octree system: brick kernels beside the table
    long long dof = 0;
    double t_submit = 0.0;
};

struct HostSlot {
    bool used = false;
    EngineJob job;
    CgState *orig = nullptr;  // the system's own state record, restored at the end
    int expect_gen = 0;       // controller generation the host waits for
    double t_admit = 0.0;
};

struct Engine {
    int device = 0, cap = 0, chunk = 8;
    double rtol = 1e-8, inner_rtol = 1e-6;
    int max_iter = 100000, max_outer = 30;
    cudaStream_t cs = nullptr;
    EngineSlot *dslots = nullptr, *hmirror = nullptr;  // mirror: 2 x cap, pinned
    tma::SysEntry *dtab = nullptr, *htab = nullptr;    // staging: 2 x cap, pinned
    unsigned int *queue = nullptr, *hhdr = nullptr;    // hhdr: 2 x 4, pinned
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr}, ev_tab[2] = {nullptr, nullptr};
    bool tab_used[2] = {false, false};
    int tab_buf = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    dim3 grid;

    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<EngineJob> pending;
    std::deque<pb_engine_result> results;
    std::vector<HostSlot> slots;
    bool stop = false;
    pb_status err = PB_OK;
    char errmsg[256] = {0};
    long long next_ticket = 1;
    long long replays = 0;
    int active = 0;
};

void engine_fail(Engine *e, const char *what, cudaError_t ce) {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->err == PB_OK) {
        e->err = PB_ERR_CUDA;
        snprintf(e->errmsg, sizeof(e->errmsg), "engine: %s: %s", what, cudaGetErrorString(ce));
    }
    e->cv_done.notify_all();
}

#define ENG_TRY(call, what)                    \
    do {                                       \
        cudaError_t ce_ = (call);              \
        if (ce_ != cudaSuccess) {              \
            engine_fail(e, what, ce_);         \
            return false;                      \
        }                                      \
    } while (0)

// queue the start of a solve in slot q: phi = boundary values, initial true
// residual, first refinement decision
bool engine_install(Engine *e, int q) {
    HostSlot &hs = e->slots[q];
    pb_system *sys = hs.job.sys;
    const GridGeo &g = sys->g->geo;
    ENG_TRY(cudaStreamWaitEvent(e->cs, hs.job.ready, 0), "waiting for the submitted system");
    hs.orig = sys->st;
    sys->st = &e->dslots[q].st;
    hs.expect_gen = 1;
    ENG_TRY(cudaMemsetAsync(e->dslots + q, 0, sizeof(EngineSlot), e->cs), "slot reset");
    ENG_TRY(cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * g.N, cudaMemcpyDeviceToDevice, e->cs),
            "initial iterate");
    if ((hs.job.oct ? oct_engine_residual(sys, e->cs) : residual(sys, true, e->cs)) != PB_OK) {
        engine_fail(e, "initial residual", cudaGetLastError());
        return false;
    }
    const size_t b32 = sizeof(float) * (size_t)sys->pad.Np;
    ENG_TRY(cudaMemsetAsync(sys->d32, 0, b32, e->cs), "correction reset");
    ENG_TRY(cudaMemsetAsync(sys->pa32, 0, b32, e->cs), "direction reset");
    k_ir_step<<<1, 32, 0, e->cs>>>(e->dslots + q, 1, hs.job.ticket, e->rtol, e->inner_rtol,
                                   e->max_iter, e->max_outer);
    ENG_TRY(cudaGetLastError(), "refinement step launch");
    note_launch(2);
    return true;
}

// queue slot q's refinement step after an inner solve ended; aborted: the
// inner solve was stopped by a device-side wait limit (status 3), so its
// incomplete correction is not promoted (k_ir_step then ends the solve)
bool engine_refine(Engine *e, int q, bool aborted) {
    HostSlot &hs = e->slots[q];
    pb_system *sys = hs.job.sys;
    const GridGeo &g = sys->g->geo;
    if (aborted) {
        // no promotion
    } else if (hs.job.oct) {
        if (oct_engine_promote(sys, e->cs) != PB_OK) {
            engine_fail(e, "promotion", cudaGetLastError());
            return false;
        }
    } else {
        k_promote<float><<<cdiv(g.N, 256), 256, 0, e->cs>>>(sys->phi, sys->d32, g, sys->pad);
        ENG_TRY(cudaGetLastError(), "promotion launch");
    }
    if ((hs.job.oct ? oct_engine_residual(sys, e->cs) : residual(sys, true, e->cs)) != PB_OK) {
        engine_fail(e, "true residual", cudaGetLastError());
        return false;
    }
    const size_t b32 = sizeof(float) * (size_t)sys->pad.Np;
    ENG_TRY(cudaMemsetAsync(sys->d32, 0, b32, e->cs), "correction reset");
    ENG_TRY(cudaMemsetAsync(sys->pa32, 0, b32, e->cs), "direction reset");
    k_ir_step<<<1, 32, 0, e->cs>>>(e->dslots + q, 0, hs.job.ticket, e->rtol, e->inner_rtol,
                                   e->max_iter, e->max_outer);
    ENG_TRY(cudaGetLastError(), "refinement step launch");
    note_launch(3);
    hs.expect_gen += 1;
    return true;
}

// rewrite the device launch table from the occupied slots (stream-ordered
// after every replay already queued)
bool engine_upload_table(Engine *e) {
    const int b = e->tab_buf;
    if (e->tab_used[b]) ENG_TRY(cudaEventSynchronize(e->ev_tab[b]), "table staging reuse");
    tma::SysEntry *h = e->htab + (size_t)b * e->cap;
    int total = 0;
    for (int q = 0; q < e->cap; ++q) {
        tma::SysEntry &en = h[q];
        const HostSlot &hs = e->slots[q];
        if (hs.used && !hs.job.oct) {
            const TmaState *ts = (const TmaState *)hs.job.sys->tma;
            en = ts->host;
            // the tile width of the maps the entry holds (the job's, set at
            // submission)
            tma_entry_geometry(en, hs.job.sys->pad, hs.job.kc, ts->tw);
        } else {  // free slot, or an octree system (solved beside the table)
            memset(&en, 0, sizeof(en));
            en.nitems = 0;
        }
        en.st = &e->dslots[q].st;
        en.item_base = total;
        total += en.nitems;
    }
    unsigned int *hdr = e->hhdr + 4 * b;
    hdr[2] = (unsigned int)e->cap;
    hdr[3] = (unsigned int)total;
    ENG_TRY(cudaMemcpyAsync(e->dtab, h, sizeof(tma::SysEntry) * e->cap, cudaMemcpyHostToDevice, e->cs),
            "table upload");
    ENG_TRY(cudaMemcpyAsync(e->queue + 2, hdr + 2, 2 * sizeof(unsigned int), cudaMemcpyHostToDevice,
                            e->cs),
            "table size upload");
    ENG_TRY(cudaEventRecord(e->ev_tab[b], e->cs), "table event");
    e->tab_used[b] = true;
    e->tab_buf ^= 1;
    return true;
}

// a slot's solve ended: report it and free the slot
void engine_complete(Engine *e, int q, const EngineSlot &m) {
    HostSlot &hs = e->slots[q];
    pb_system *sys = hs.job.sys;
    const GridGeo &g = sys->g->geo;
    sys->st = hs.orig;
    sys->fnorm2 = m.ctl.fn2;
    sys->solved = 1;
    pb_engine_result r{};
    r.ticket = hs.job.ticket;
    r.system = sys;
    r.stats.status = m.ctl.status;
    r.stats.iters_inner = m.ctl.iters;
    r.stats.iters_outer = m.ctl.outer;
    r.stats.kc = hs.job.oct ? 0 : hs.job.kc + 1000 + 10000 * hs.job.tw;
    r.stats.true_rel_res = m.ctl.fn2 > 0.0 ? sqrt(m.ctl.res2 / m.ctl.fn2) : 0.0;
    r.stats.dof = hs.job.dof;
    r.stats.model_bytes = (long long)m.ctl.iters * r.stats.dof * (8 * 4 + 2) +
                          (long long)m.ctl.outer * g.N * 64;
    r.t_submit = hs.job.t_submit;
    r.t_admit = hs.t_admit;
    r.t_done = now_s();
    r.stats.seconds = r.t_done - r.t_admit;
    cudaEventDestroy(hs.job.ready);
    hs = HostSlot();
    std::lock_guard<std::mutex> lk(e->mu);
    e->results.push_back(r);
    e->active -= 1;
    e->cv_done.notify_all();
}

bool engine_issue(Engine *e, int mb) {
    ENG_TRY(cudaGraphLaunch(e->exec, e->cs), "replay");
    note_launch(2 * e->chunk);
    // octree systems: the same number of iterations with their brick kernels
    for (int q = 0; q < e->cap; ++q) {
        const HostSlot &hs = e->slots[q];
        if (!hs.used || !hs.job.oct) continue;
        if (oct_engine_iterations(hs.job.sys, e->chunk, e->cs) != PB_OK) {
            engine_fail(e, "octree iterations", cudaGetLastError());
            return false;
        }
    }
    ENG_TRY(cudaMemcpyAsync(e->hmirror + (size_t)mb * e->cap, e->dslots, sizeof(EngineSlot) * e->cap,
                            cudaMemcpyDeviceToHost, e->cs),
            "state mirror");
    ENG_TRY(cudaEventRecord(e->ev_chunk[mb], e->cs), "replay event");
    e->replays += 1;
    return true;
}

// handle the state mirror of one finished replay
bool engine_process(Engine *e, int mb, bool *changed) {
    const EngineSlot *m = e->hmirror + (size_t)mb * e->cap;
    for (int q = 0; q < e->cap; ++q) {
        HostSlot &hs = e->slots[q];
        if (!hs.used) continue;
        const EngineSlot &ms = m[q];
        // a mirror taken before this occupant's latest step is stale
        if (ms.ctl.ticket != hs.job.ticket || ms.ctl.gen != hs.expect_gen) continue;
        if (ms.ctl.final_) {
            engine_complete(e, q, ms);
            *changed = true;
        } else if (ms.st.done) {
            if (!engine_refine(e, q, ms.st.status == 3)) return false;
        }
    }
    return true;
}

void engine_pump(Engine *e) {
    if (cudaSetDevice(e->device) != cudaSuccess) {
        engine_fail(e, "cudaSetDevice", cudaGetLastError());
        return;
    }
    int inflight[2];
    int n_inflight = 0, next_mb = 0;
    bool changed = false;
    for (;;) {
        // admit waiting jobs into free slots
        std::vector<int> fresh;
        {
            std::unique_lock<std::mutex> lk(e->mu);
            if (e->err != PB_OK) break;
            if (e->stop) break;
            for (int q = 0; q < e->cap && !e->pending.empty(); ++q) {
                if (e->slots[q].used) continue;
                e->slots[q].used = true;
                e->slots[q].job = e->pending.front();
                e->slots[q].t_admit = now_s();
                e->pending.pop_front();
                e->active += 1;
                fresh.push_back(q);
            }
            if (fresh.empty() && e->active == 0 && n_inflight == 0) {
                e->cv_work.wait(lk, [&] { return e->stop || !e->pending.empty(); });
                continue;
            }
        }
        bool ok = true;
        for (int q : fresh) ok = ok && engine_install(e, q);
        if (!ok) break;
        if (!fresh.empty()) changed = true;
        if (changed) {
            if (!engine_upload_table(e)) break;
            changed = false;
        }
        if (e->active > 0 && n_inflight < 2) {
            if (!engine_issue(e, next_mb)) break;
            inflight[n_inflight++] = next_mb;
            next_mb ^= 1;
            if (n_inflight < 2) continue;  // keep two replays in flight
        }
        if (n_inflight == 0) continue;
        const int mb = inflight[0];
        cudaError_t ce = cudaEventSynchronize(e->ev_chunk[mb]);
        if (ce != cudaSuccess) {
            engine_fail(e, "replay", ce);
            break;
        }
        inflight[0] = inflight[1];
        n_inflight -= 1;
        if (!engine_process(e, mb, &changed)) break;
    }
    cudaStreamSynchronize(e->cs);
    // hand back the systems still in the table, then fail what is left
    std::lock_guard<std::mutex> lk(e->mu);
    for (HostSlot &hs : e->slots) {
        if (!hs.used) continue;
        hs.job.sys->st = hs.orig;
        pb_engine_result r{};
        r.ticket = hs.job.ticket;
        r.system = hs.job.sys;
        r.stats.status = e->err != PB_OK ? e->err : PB_ERR_STATE;
        r.t_submit = hs.job.t_submit;
        r.t_admit = hs.t_admit;
        r.t_done = now_s();
        e->results.push_back(r);
        cudaEventDestroy(hs.job.ready);
        hs = HostSlot();
    }
    for (EngineJob &j : e->pending) {
        pb_engine_result r{};
        r.ticket = j.ticket;
        r.system = j.sys;
        r.stats.status = e->err != PB_OK ? e->err : PB_ERR_STATE;
        r.t_submit = j.t_submit;
        r.t_done = now_s();
        e->results.push_back(r);
        cudaEventDestroy(j.ready);
    }
    e->pending.clear();
    e->active = 0;
    e->cv_done.notify_all();
}

#undef ENG_TRY

void engine_release(Engine *e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->cs) cudaStreamSynchronize(e->cs);
    for (cudaEvent_t ev : {e->ev_chunk[0], e->ev_chunk[1], e->ev_tab[0], e->ev_tab[1]})
        if (ev) cudaEventDestroy(ev);
    dfree(e->dslots, e->cs);
    dfree(e->dtab, e->cs);
    dfree(e->queue, e->cs);
    if (e->cs) {
        cudaStreamSynchronize(e->cs);
        cudaStreamDestroy(e->cs);
    }
    if (e->hmirror) cudaFreeHost(e->hmirror);
    if (e->htab) cudaFreeHost(e->htab);
    if (e->hhdr) cudaFreeHost(e->hhdr);
    delete e;
}

}  // namespace

pb_status engine_create(int device, int capacity, const pb_solve_opts *o, pb_engine **out) {
    Engine *e = new (std::nothrow) Engine();
    if (!e) return PB_ERR_OOM;
    e->device = device;
    e->cap = capacity;
    if (o) {
        if (o->rtol > 0.0) e->rtol = o->rtol;
        if (o->inner_rtol > 0.0) e->inner_rtol = o->inner_rtol;
        if (o->max_iter > 0) e->max_iter = o->max_iter;
        if (o->max_outer > 0) e->max_outer = o->max_outer;
    }
    e->slots.resize(capacity);
    auto bail = [&](pb_status rc, const char *what) {
        cudaError_t ce = cudaGetLastError();
        set_error("engine creation failed at %s: %s", what, cudaGetErrorString(ce));
        engine_release(e);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(PB_ERR_CUDA, "stream");
    for (cudaEvent_t *ev : {&e->ev_chunk[0], &e->ev_chunk[1], &e->ev_tab[0], &e->ev_tab[1]})
        if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(PB_ERR_CUDA, "events");
    e->dslots = (EngineSlot *)dalloc(sizeof(EngineSlot) * capacity, e->cs);
    e->dtab = (tma::SysEntry *)dalloc(sizeof(tma::SysEntry) * capacity, e->cs);
    e->queue = (unsigned int *)dalloc(4 * sizeof(unsigned int), e->cs);
    if (!e->dslots || !e->dtab || !e->queue) return bail(PB_ERR_OOM, "device allocation");
    if (cudaMallocHost((void **)&e->hmirror, 2 * sizeof(EngineSlot) * capacity) != cudaSuccess ||
        cudaMallocHost((void **)&e->htab, 2 * sizeof(tma::SysEntry) * capacity) != cudaSuccess ||
        cudaMallocHost((void **)&e->hhdr, 8 * sizeof(unsigned int)) != cudaSuccess)
        return bail(PB_ERR_OOM, "pinned host allocation");
    memset(e->hhdr, 0, 8 * sizeof(unsigned int));
    if (cudaMemsetAsync(e->dslots, 0, sizeof(EngineSlot) * capacity, e->cs) != cudaSuccess ||
        cudaMemsetAsync(e->dtab, 0, sizeof(tma::SysEntry) * capacity, e->cs) != cudaSuccess ||
        cudaMemsetAsync(e->queue, 0, 4 * sizeof(unsigned int), e->cs) != cudaSuccess)
        return bail(PB_ERR_CUDA, "initialisation");
    if (tma_prepare<MODE_P>() != PB_OK || tma_prepare<MODE_U>() != PB_OK)
        return bail(PB_ERR_CUDA, "kernel attributes");
    e->grid = tma_grid(PadGeo{}, 8);
    // one replay: `chunk` PCG iterations of whatever the table holds
    if (cudaStreamBeginCapture(e->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail(PB_ERR_CUDA, "capture");
    for (int c = 0; c < e->chunk; ++c) {
        tma_launch<MODE_P>(e->dtab, -1, 0, e->queue, e->grid, e->cs);
        tma_launch<MODE_U>(e->dtab, -1, 0, e->queue, e->grid, e->cs);
    }
    if (cudaStreamEndCapture(e->cs, &e->graph) != cudaSuccess ||
        cudaGraphInstantiate(&e->exec, e->graph, 0) != cudaSuccess)
        return bail(PB_ERR_CUDA, "graph instantiation");
    if (cudaStreamSynchronize(e->cs) != cudaSuccess) return bail(PB_ERR_CUDA, "set-up");
    try {
        e->th = std::thread(engine_pump, e);
    } catch (...) {
        set_error("engine thread could not start");
        engine_release(e);
        return PB_ERR_STATE;
    }
    *out = reinterpret_cast<pb_engine *>(e);
    return PB_OK;
}

pb_status engine_submit(pb_engine *eh, pb_system *sys, cudaStream_t s, long long *ticket) {
    Engine *e = reinterpret_cast<Engine *>(eh);
    if (sys->g->device != e->device) {
        set_error("the system lives on device %d, the engine on device %d", sys->g->device, e->device);
        return PB_ERR_ARG;
    }
    EngineJob j;
    j.sys = sys;
    pb_status rc = PB_OK;
    if (sys->g->is_oct) {
        if ((rc = oct_engine_prepare(sys, s)) != PB_OK) return rc;
        j.oct = true;
        j.kc = 0;
        j.dof = sys->os->nunk;
    } else {
        if ((rc = ensure_solver_ws(sys, PB_MIXED, s)) != PB_OK) return rc;
        if ((rc = build_tma_state(sys)) != PB_OK) return rc;
        Tuning tune;
        if ((rc = autotune(sys, PB_MIXED, s, &tune)) != PB_OK) return rc;
        j.kc = tune.variant == 1 ? std::max(tune.kc, 4) : 8;
        j.tw = tune.variant == 1 ? tune.tw : tma::TWDEF;
        // the entry the table copies holds the maps of this tile width
        if ((rc = tma_set_tile(sys, j.tw)) != PB_OK) return rc;
        const GridGeo &gg = sys->g->geo;
        j.dof = (long long)(gg.nx - 2) * (gg.ny - 2) * (gg.nz - 2);
    }
    j.t_submit = now_s();
    PB_CUDA_TRY(cudaEventCreateWithFlags(&j.ready, cudaEventDisableTiming));
    cudaError_t ce = cudaEventRecord(j.ready, s);
    if (ce != cudaSuccess) {
        cudaEventDestroy(j.ready);
        set_error("recording the submission event failed: %s", cudaGetErrorString(ce));
        return PB_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (e->err != PB_OK || e->stop) {
            cudaEventDestroy(j.ready);
            set_error("%s", e->err != PB_OK ? e->errmsg : "engine is shutting down");
            return e->err != PB_OK ? e->err : PB_ERR_STATE;
        }
        for (const HostSlot &hs : e->slots)
            if (hs.used && hs.job.sys == sys) {
                cudaEventDestroy(j.ready);
                set_error("the system is already being solved by the engine");
                return PB_ERR_ARG;
            }
        for (const EngineJob &p : e->pending)
            if (p.sys == sys) {
                cudaEventDestroy(j.ready);
                set_error("the system is already waiting in the engine");
                return PB_ERR_ARG;
            }
        j.ticket = e->next_ticket++;
        e->pending.push_back(j);
        *ticket = j.ticket;
    }
    e->cv_work.notify_all();
    return PB_OK;
}

pb_status engine_wait(pb_engine *eh, double timeout_s, pb_engine_result *out, int max_out, int *n_out) {
    Engine *e = reinterpret_cast<Engine *>(eh);
    std::unique_lock<std::mutex> lk(e->mu);
    auto ready = [&] { return !e->results.empty() || e->err != PB_OK; };
    if (timeout_s > 0.0 && !ready())
        e->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    int n = 0;
    while (n < max_out && !e->results.empty()) {
        out[n++] = e->results.front();
        e->results.pop_front();
    }
    *n_out = n;
    if (e->err != PB_OK && n == 0) {
        set_error("%s", e->errmsg);
        return e->err;
    }
    return PB_OK;
}

pb_status engine_query(pb_engine *eh, int *n_pending, int *n_active, long long *replays) {
    Engine *e = reinterpret_cast<Engine *>(eh);
    std::lock_guard<std::mutex> lk(e->mu);
    if (n_pending) *n_pending = (int)e->pending.size();
    if (n_active) *n_active = e->active;
    if (replays) *replays = e->replays;
    return e->err;
}

pb_status engine_destroy(pb_engine *eh) {
    Engine *e = reinterpret_cast<Engine *>(eh);
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
    }
    e->cv_work.notify_all();
    if (e->th.joinable()) e->th.join();
    engine_release(e);
    return PB_OK;
}
