// C ABI of libpbgpu (declared in include/pb.h): argument checking, handle
// lifetime, device-memory hooks and the order of the device passes.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "pb_internal.h"

namespace pbg {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static std::atomic<long long> g_launches{0};
void note_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// --------------------------------------------------------------- allocator
static std::mutex g_alloc_mu;
static pb_alloc_fn g_alloc = nullptr;
static pb_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void *dalloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    pb_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    void *p = nullptr;
    if (a) {
        p = a(ctx, bytes, (void *)s);
    } else if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) set_error("device allocation of %zu bytes failed", bytes);
    return p;
}

void dfree(void *p, cudaStream_t s) {
    if (!p) return;
    pb_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f) f(ctx, p, (void *)s);
    else cudaFreeAsync(p, s);
}

// Units: reduced potential kT/e, lengths in Angstrom (CODATA 2018 values).
static void physical_units(double T, double I, double eps_out, double *lB, double *kD) {
    const double qe = 1.602176634e-19, e0 = 8.8541878128e-12, kb = 1.380649e-23,
                 na = 6.02214076e23;
    // Bjerrum length in vacuum, metres -> Angstrom
    double bj = qe * qe / (4.0 * M_PI * e0 * kb * T) * 1e10;
    // Debye factor: k^2 = 4 pi l_B sum_j z_j^2 rho_j / eps_out, 1:1 salt,
    // rho in ions per A^3 (mol/L -> 1e-27 * N_A per A^3)
    double rho = 2.0 * I * na * 1e-27;
    *lB = bj;
    *kD = sqrt(4.0 * M_PI * bj * rho / eps_out);
}

static thread_local char g_stale[256] = "";

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        // a non-sticky error left by an earlier call must not be reported
        // as a failure of this one; keep its text for diagnostics
        cudaError_t stale = cudaGetLastError();
        if (stale != cudaSuccess)
            snprintf(g_stale, sizeof(g_stale), "%s", cudaGetErrorString(stale));
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            if (cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();
        } else {
            prev = -1;
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace pbg

using namespace pbg;

namespace pbg {
pb_status upload_atoms(pb_grid *g, const double *atoms, int loc, cudaStream_t s);
}

extern "C" {

const char *pb_last_error(void) {
    if (g_stale[0] && g_err[0]) {
        static thread_local char both[800];
        snprintf(both, sizeof(both), "%s [earlier: %s]", g_err, g_stale);
        return both;
    }
    return g_err;
}

const char *pb_version(void) { return "pbgpu 0.1 (sm_103a)"; }

pb_status pb_set_allocator(pb_alloc_fn alloc, pb_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr)) {
        set_error("pb_set_allocator: give both hooks or neither");
        return PB_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return PB_OK;
}

void pb_grid_free(pb_grid *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaStream_t s = g->stream;
    cudaStreamSynchronize(s);
    dfree(g->atoms, s);
    dfree(g->inside, s);
    dfree(g->cells.start, s);
    dfree(g->cells.atom, s);
    dfree(g->cid, s);
    dfree(g->calpha, s);
    dfree(g->crp, s);
    dfree(g->csign, s);
    dfree(g->rowstart, s);
    dfree(g->mc_w, s);
    dfree(g->mc_n, s);
    dfree(g->d_info, s);
    if (g->is_oct) oct_grid_free(g, s);
    cudaStreamSynchronize(s);
    delete g;
}

pb_status pb_build_grid(const pb_grid_spec *spec, const double *atoms, int64_t n_atoms,
                        int32_t atoms_loc, void *stream, pb_grid **out) {
    set_error("");
    if (!spec || !out || !atoms || n_atoms < 1) {
        set_error("pb_build_grid: NULL argument or no atoms");
        return PB_ERR_ARG;
    }
    *out = nullptr;
    const bool oct = spec->kind == PB_GRID_OCTREE;
    if (spec->kind != PB_GRID_UNIFORM && !oct) {
        set_error("unknown grid kind %d", spec->kind);
        return PB_ERR_ARG;
    }
    if (oct) {
        if (!(spec->h_fine > 0.0) || !(spec->h_bulk >= spec->h_fine) || !isfinite(spec->h_bulk) ||
            !(spec->refine_dist >= 0.0) || !isfinite(spec->refine_dist)) {
            set_error("octree: need 0 < h_fine <= h_bulk and refine_dist >= 0");
            return PB_ERR_ARG;
        }
        if (spec->n[0] < 0 || spec->n[0] > 1024) {
            set_error("octree: n[0] (coarse bricks per axis) out of range [0, 1024]");
            return PB_ERR_ARG;
        }
        if (spec->n[0] == 0 && (!(spec->fill > 1.0) || !isfinite(spec->fill))) {
            set_error("automatic placement needs fill > 1");
            return PB_ERR_ARG;
        }
        for (int d = 0; d < 3; ++d)
            if (spec->n[0] > 0 && !isfinite(spec->origin[d])) {
                set_error("grid origin is not finite");
                return PB_ERR_ARG;
            }
    }
    for (int d = 0; d < 3 && !oct; ++d)
        if (spec->n[d] < 3 || spec->n[d] > 4096) {
            set_error("grid size n[%d]=%d out of range [3, 4096]", d, spec->n[d]);
            return PB_ERR_ARG;
        }
    if (!oct && (long long)spec->n[0] * spec->n[1] * spec->n[2] > (1ll << 31) - 1) {
        set_error("grid has more than 2^31 nodes");
        return PB_ERR_ARG;
    }
    if (!(spec->h >= 0.0) || !isfinite(spec->h)) {
        set_error("grid spacing h must be >= 0 and finite");
        return PB_ERR_ARG;
    }
    if (oct) {
        // checked above
    } else if (spec->h == 0.0) {
        if (!(spec->fill > 1.0) || !isfinite(spec->fill)) {
            set_error("automatic placement needs fill > 1");
            return PB_ERR_ARG;
        }
        if (spec->n[0] != spec->n[1] || spec->n[1] != spec->n[2]) {
            set_error("automatic placement needs a cubic grid (n[0]==n[1]==n[2])");
            return PB_ERR_ARG;
        }
    } else {
        for (int d = 0; d < 3; ++d)
            if (!isfinite(spec->origin[d])) {
                set_error("grid origin is not finite");
                return PB_ERR_ARG;
            }
    }
    if (atoms_loc != PB_HOST && atoms_loc != PB_DEVICE) {
        set_error("atoms_loc must be PB_HOST or PB_DEVICE");
        return PB_ERR_ARG;
    }
    if (atoms_loc == PB_HOST) {
        for (int64_t i = 0; i < n_atoms; ++i) {
            const double *p = atoms + 5 * i;
            for (int d = 0; d < 5; ++d)
                if (!isfinite(p[d])) {
                    set_error("atom %lld has a non-finite value", (long long)i);
                    return PB_ERR_ARG;
                }
            if (!(p[3] > 0.0)) {
                set_error("atom %lld has a non-positive radius", (long long)i);
                return PB_ERR_ARG;
            }
            if (fabs(p[4]) > 100.0) {
                set_error("atom %lld has |q| > 100 e", (long long)i);
                return PB_ERR_ARG;
            }
        }
    }
    int cur = 0;
    cudaGetDevice(&cur);
    DeviceGuard dg0(cur);
    cudaStream_t s = (cudaStream_t)stream;
    pb_grid *g = new (std::nothrow) pb_grid();
    if (!g) return PB_ERR_OOM;
    cudaGetDevice(&g->device);
    g->stream = s;
    g->na = n_atoms;
    g->d_info = (BuildInfo *)dalloc(sizeof(BuildInfo), s);
    if (!g->d_info) {
        pb_grid_free(g);
        return PB_ERR_OOM;
    }
    pb_status st = upload_atoms(g, atoms, atoms_loc, s);
    if (st == PB_OK) st = oct ? oct_build(g, spec, s) : grid_build(g, spec, s);
    if (st != PB_OK) {
        pb_grid_free(g);
        return st;
    }
    *out = g;
    return PB_OK;
}

pb_status pb_grid_info_get(const pb_grid *g, pb_grid_info *info) {
    if (!g || !info) {
        set_error("pb_grid_info_get: NULL argument");
        return PB_ERR_ARG;
    }
    info->n[0] = g->geo.nx;
    info->n[1] = g->geo.ny;
    info->n[2] = g->geo.nz;
    for (int d = 0; d < 3; ++d) info->origin[d] = g->geo.o[d];
    info->h = g->geo.h;
    info->n_nodes = g->geo.N;
    info->n_atoms = g->na;
    info->n_cross = g->ncross;
    info->n_flux = g->nflux;
    info->n_inside = g->ninside;
    info->kind = g->is_oct ? PB_GRID_OCTREE : PB_GRID_UNIFORM;
    info->n_levels = g->is_oct ? g->ot.Lmax + 1 : 1;
    info->n_bricks = g->is_oct ? g->ot.nb : 0;
    if (g->is_oct)
        for (int d = 0; d < 3; ++d) info->n[d] = g->ot.NL + 1;
    return PB_OK;
}

void pb_system_free(pb_system *s) {
    if (!s) return;
    DeviceGuard dg(s->g->device);
    cudaStream_t st = s->stream;
    cudaStreamSynchronize(st);
    void *ptrs[] = {s->W[0], s->W[1], s->W[2], s->diag, s->rhs, s->bc, s->phi, s->code, s->w32[0], s->w32[1], s->w32[2],
                    s->z32, s->pa32, s->pb32, s->d32, s->z64, s->pa64, s->pb64, s->x64,
                    s->r64, s->q64, s->op64[0], s->op64[1], s->op64[2], s->op64[3], s->op64[4],
                    s->partials, s->queue, s->st, s->Phi, s->Psi, s->eacc, s->PsiN};
    for (void *p : ptrs) dfree(p, st);
    oct_system_free(s, st);
    cudaStreamSynchronize(st);
    free_tma_state(s);
    if (s->h_st) cudaFreeHost(s->h_st);
    if (s->h_energy) cudaFreeHost(s->h_energy);
    delete s;
}

pb_status pb_assemble_coeffs(pb_grid *g, const pb_params *params, void *stream, pb_system **out) {
    set_error("");
    if (!g || !params || !out) {
        set_error("pb_assemble_coeffs: NULL argument");
        return PB_ERR_ARG;
    }
    *out = nullptr;
    const pb_params &p = *params;
    if (!(p.eps_in > 0.0) || !(p.eps_out > 0.0) || !isfinite(p.eps_in) || !isfinite(p.eps_out)) {
        set_error("permittivities must be positive and finite");
        return PB_ERR_ARG;
    }
    if (!(p.ionic_strength_M >= 0.0) || !isfinite(p.ionic_strength_M)) {
        set_error("ionic strength must be >= 0");
        return PB_ERR_ARG;
    }
    if (!(p.temperature_K > 0.0) || !isfinite(p.temperature_K)) {
        set_error("temperature must be > 0");
        return PB_ERR_ARG;
    }
    if (p.bc != PB_BC_ZERO && p.bc != PB_BC_COULOMB && p.bc != PB_BC_DH) {
        set_error("unknown boundary condition %d", p.bc);
        return PB_ERR_ARG;
    }
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    pb_system *sys = new (std::nothrow) pb_system();
    if (!sys) return PB_ERR_OOM;
    sys->g = g;
    sys->stream = s;
    sys->p = p;
    physical_units(p.temperature_K, p.ionic_strength_M, p.eps_out, &sys->lB, &sys->kD);
    const double h = g->geo.h;
    sys->kap_s = p.eps_out * sys->kD * sys->kD * h * h * h;
    pb_status st = PB_OK;
    sys->eacc = (EnergyAcc *)dalloc(sizeof(EnergyAcc), s);
    if (!sys->eacc) st = PB_ERR_OOM;
    if (st == PB_OK && cudaMemsetAsync(sys->eacc, 0, sizeof(EnergyAcc), s) != cudaSuccess)
        st = PB_ERR_CUDA;
    if (st == PB_OK && cudaMallocHost((void **)&sys->h_energy, sizeof(pb_energy_terms)) != cudaSuccess) {
        set_error("pinned host allocation failed");
        st = PB_ERR_OOM;
    }
    if (g->is_oct) {
        if (st == PB_OK) st = oct_assemble(sys, s);
    } else {
        if (st == PB_OK) st = assemble(sys, s);
        if (st == PB_OK) st = nbody_boundary(sys, s);
        if (st == PB_OK) st = deposit_rhs(sys, s);
    }
    if (st != PB_OK) {
        pb_system_free(sys);
        return st;
    }
    *out = sys;
    return PB_OK;
}

pb_status pb_coulomb_terms(pb_system *s, int32_t which, void *stream) {
    set_error("");
    if (!s || (which & ~PB_CT_ALL) || which == 0) {
        set_error("pb_coulomb_terms: NULL system or bad selector");
        return PB_ERR_ARG;
    }
    DeviceGuard dg(s->g->device);
    cudaStream_t st = (cudaStream_t)stream;
    pb_status rc = PB_OK;
    if (which & PB_CT_BOUNDARY) {
        if (s->g->is_oct) {
            rc = oct_boundary_rhs(s, st);
        } else {
            rc = nbody_boundary(s, st);
            if (rc == PB_OK) rc = deposit_rhs(s, st);
        }
        if (rc == PB_OK) s->solved = 0;
    }
    if (rc == PB_OK && (which & PB_CT_SURFACE)) {
        rc = nbody_surface(s, st);
        if (rc == PB_OK) s->have_surface = 1;
    }
    if (rc == PB_OK && (which & PB_CT_PAIRS)) {
        rc = nbody_pairs(s, st);
        if (rc == PB_OK) s->have_pairs = 1;
    }
    return rc;
}

static pb_status check_opts(const pb_solve_opts *o) {
    if (!o) {
        set_error("NULL solve options");
        return PB_ERR_ARG;
    }
    if (o->precision != PB_FP64 && o->precision != PB_MIXED) {
        set_error("precision must be PB_FP64 or PB_MIXED");
        return PB_ERR_ARG;
    }
    if (!(o->rtol >= 0.0) || !(o->inner_rtol >= 0.0) || !(o->time_budget_s >= 0.0) ||
        o->max_iter < 0 || o->max_outer < 0) {
        set_error("invalid solve options");
        return PB_ERR_ARG;
    }
    return PB_OK;
}

pb_status pb_solve(pb_system *s, const pb_solve_opts *opts, double *phi_dev, void *stream,
                   pb_solve_stats *stats) {
    set_error("");
    if (!s) {
        set_error("pb_solve: NULL system");
        return PB_ERR_ARG;
    }
    pb_status rc = check_opts(opts);
    if (rc != PB_OK) return rc;
    DeviceGuard dg(s->g->device);
    cudaStream_t st = (cudaStream_t)stream;
    rc = s->g->is_oct ? oct_solve(s, opts, st, stats) : solve(s, opts, st, stats);
    if (rc == PB_ERR_NOCONV) set_error("solver stopped before reaching rtol");
    // a device-side wait limit reports its own message
    if (rc == PB_ERR_TIMEOUT && !g_err[0]) set_error("solver exceeded its time budget");
    if ((rc == PB_OK || rc == PB_ERR_NOCONV) && phi_dev) {
        PB_CUDA_TRY(cudaMemcpyAsync(phi_dev, s->phi, sizeof(double) * s->g->geo.N,
                                    cudaMemcpyDeviceToDevice, st));
    }
    return rc;
}

pb_status pb_energy(pb_system *s, void *stream, pb_energy_terms *out) {
    set_error("");
    if (!s || !out) {
        set_error("pb_energy: NULL argument");
        return PB_ERR_ARG;
    }
    if (!s->solved || !s->have_surface || !s->have_pairs) {
        set_error("pb_energy needs pb_solve and pb_coulomb_terms(SURFACE|PAIRS) first");
        return PB_ERR_STATE;
    }
    DeviceGuard dg(s->g->device);
    if (s->g->is_oct) return oct_energy(s, (cudaStream_t)stream, out);
    return energy(s, (cudaStream_t)stream, out);
}

pb_status pb_get_phi(pb_system *s, double *dst, int32_t dst_loc, void *stream) {
    if (!s || !dst) {
        set_error("pb_get_phi: NULL argument");
        return PB_ERR_ARG;
    }
    return pb_get_array(s->g, s, PB_ARR_PHI, dst, sizeof(double) * s->g->geo.N, dst_loc, stream);
}

pb_status pb_get_array(const pb_grid *g, const pb_system *s, int32_t which, void *dst, size_t bytes,
                       int32_t dst_loc, void *stream) {
    set_error("");
    if (s && !g) g = s->g;
    if (!g || !dst || which < 0 || which >= PB_ARR_COUNT) {
        set_error("pb_get_array: NULL argument or bad array id");
        return PB_ERR_ARG;
    }
    if (dst_loc != PB_HOST && dst_loc != PB_DEVICE) {
        set_error("dst_loc must be PB_HOST or PB_DEVICE");
        return PB_ERR_ARG;
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = g->geo.N, nc = g->ncross;
    const void *src = nullptr;
    size_t need = 0;
    bool tmp = false;
    switch (which) {
        case PB_ARR_INSIDE: src = g->inside; need = N; break;
        case PB_ARR_CROSS_ID: src = g->cid; need = 8 * nc; break;
        case PB_ARR_CROSS_ALPHA: src = g->calpha; need = 8 * nc; break;
        case PB_ARR_CROSS_RP: src = g->crp; need = 24 * nc; break;
        case PB_ARR_CROSS_SIGN: src = g->csign; need = nc; break;
        case PB_ARR_OCT_BRICKS:
        case PB_ARR_OCT_KIND:
            if (!g->is_oct) {
                set_error("array %d exists on octree grids only", which);
                return PB_ERR_ARG;
            }
            src = which == PB_ARR_OCT_BRICKS ? (const void *)g->ot.blow : (const void *)g->ot.okind;
            need = which == PB_ARR_OCT_BRICKS ? 16 * g->ot.nb : g->ot.N;
            break;
        default: break;
    }
    if (which >= PB_ARR_WX && which <= PB_ARR_PSI_SURF) {
        if (!s) {
            set_error("array %d needs a system", which);
            return PB_ERR_ARG;
        }
        switch (which) {
            case PB_ARR_WX: src = s->W[0]; need = 8 * N; break;
            case PB_ARR_WY: src = s->W[1]; need = 8 * N; break;
            case PB_ARR_WZ: src = s->W[2]; need = 8 * N; break;
            case PB_ARR_DIAG: src = s->diag; need = 8 * N; break;
            case PB_ARR_RHS: src = s->rhs; need = 8 * N; break;
            case PB_ARR_BC: src = s->bc; need = 8 * N; break;
            case PB_ARR_PHI:
                if (!s->solved) {
                    set_error("no solution yet");
                    return PB_ERR_STATE;
                }
                src = s->phi;
                need = 8 * N;
                break;
            case PB_ARR_PHI_SURF:
            case PB_ARR_PSI_SURF:
                if (!s->have_surface) {
                    set_error("surface Coulomb terms not computed");
                    return PB_ERR_STATE;
                }
                src = which == PB_ARR_PHI_SURF ? s->Phi : s->Psi;
                need = 8 * nc;
                break;
            case PB_ARR_KAPPA: {
                need = 8 * N;
                double *t = (double *)dalloc(need, st);
                if (!t) return PB_ERR_OOM;
                pb_status rc = g->is_oct ? oct_fill_kappa(s, t, st) : fill_kappa(s, t, st);
                if (rc != PB_OK) return rc;
                src = t;
                tmp = true;
                break;
            }
            default: break;
        }
    }
    if (which == PB_ARR_MC_WEIGHT || which == PB_ARR_MC_NORMAL) {
        src = which == PB_ARR_MC_WEIGHT ? g->mc_w : g->mc_n;
        need = (which == PB_ARR_MC_NORMAL ? 24 : 8) * nc;
    }
    if (which == PB_ARR_PSI_N) {
        if (!s) {
            set_error("array %d needs a system", which);
            return PB_ERR_ARG;
        }
        if (!s->have_surface || !s->PsiN) {
            set_error("surface Coulomb terms not computed");
            return PB_ERR_STATE;
        }
        src = s->PsiN;
        need = 8 * nc;
    }
    if (bytes < need) {
        set_error("destination too small: %zu < %zu bytes", bytes, need);
        if (tmp) dfree((void *)src, st);
        return PB_ERR_ARG;
    }
    if (need > 0) {
        cudaError_t e = cudaMemcpyAsync(dst, src, need,
                                        dst_loc == PB_HOST ? cudaMemcpyDeviceToHost
                                                           : cudaMemcpyDeviceToDevice,
                                        st);
        if (e == cudaSuccess && dst_loc == PB_HOST) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("copy failed: %s", cudaGetErrorString(e));
            if (tmp) dfree((void *)src, st);
            return PB_ERR_CUDA;
        }
    }
    if (tmp) dfree((void *)src, st);
    return PB_OK;
}

pb_status pb_apply(pb_system *s, int32_t precision, const void *x, void *y, void *stream) {
    set_error("");
    if (!s || !x || !y || (precision != PB_FP64 && precision != PB_MIXED)) {
        set_error("pb_apply: NULL argument or bad precision");
        return PB_ERR_ARG;
    }
    DeviceGuard dg(s->g->device);
    if (s->g->is_oct) return oct_apply(s, precision, x, y, (cudaStream_t)stream);
    return apply_op(s, precision, x, y, (cudaStream_t)stream);
}

pb_status pb_solve_batch(pb_system *const *systems, int32_t n, const pb_solve_opts *opts,
                         void *stream, pb_solve_stats *stats) {
    set_error("");
    if (!systems || n < 0 || (n > 0 && !stats)) {
        set_error("pb_solve_batch: NULL argument");
        return PB_ERR_ARG;
    }
    pb_status rc = check_opts(opts);
    if (rc != PB_OK) return rc;
    for (int i = 0; i < n; ++i) {
        if (!systems[i]) {
            set_error("pb_solve_batch: system %d is NULL", i);
            return PB_ERR_ARG;
        }
        if (systems[i]->g->device != systems[0]->g->device) {
            set_error("pb_solve_batch: systems live on different devices");
            return PB_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (systems[j] == systems[i]) {
                set_error("pb_solve_batch: system %d appears twice", i);
                return PB_ERR_ARG;
            }
    }
    if (n == 0) return PB_OK;
    DeviceGuard dg(systems[0]->g->device);
    if (opts->precision == PB_MIXED) {
        pb_status r = solve_batch(systems, n, opts, (cudaStream_t)stream, stats);
        if (r == PB_ERR_NOCONV) set_error("a system stopped before reaching rtol");
        if (r == PB_ERR_TIMEOUT && !g_err[0]) set_error("the batch exceeded its time budget");
        return r;
    }
    // FP64: one plain PCG after the other
    pb_status worst = PB_OK;
    for (int i = 0; i < n; ++i) {
        pb_status r = pb_solve(systems[i], opts, nullptr, stream, &stats[i]);
        if (r == PB_ERR_CUDA || r == PB_ERR_OOM) return r;
        if (r != PB_OK) worst = r;
    }
    return worst;
}

pb_status pb_engine_create(int32_t device, int32_t capacity, const pb_solve_opts *opts,
                           pb_engine **out) {
    set_error("");
    if (!out || capacity < 1 || capacity > 4096) {
        set_error("pb_engine_create: NULL output or capacity outside 1..4096");
        return PB_ERR_ARG;
    }
    *out = nullptr;
    if (opts) {
        pb_status rc = check_opts(opts);
        if (rc != PB_OK) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("pb_engine_create: no CUDA device %d", device);
        return PB_ERR_ARG;
    }
    DeviceGuard dg(device);
    return engine_create(device, capacity, opts, out);
}

pb_status pb_engine_submit(pb_engine *e, pb_system *s, void *stream, int64_t *ticket) {
    set_error("");
    if (!e || !s || !ticket) {
        set_error("pb_engine_submit: NULL argument");
        return PB_ERR_ARG;
    }
    DeviceGuard dg(s->g->device);
    long long t = 0;
    pb_status rc = engine_submit(e, s, (cudaStream_t)stream, &t);
    *ticket = t;
    return rc;
}

pb_status pb_engine_wait(pb_engine *e, double timeout_s, pb_engine_result *out, int32_t max_out,
                         int32_t *n_out) {
    set_error("");
    if (!e || !n_out || max_out < 0 || (max_out > 0 && !out) || !(timeout_s >= 0.0)) {
        set_error("pb_engine_wait: bad argument");
        return PB_ERR_ARG;
    }
    int n = 0;
    pb_status rc = engine_wait(e, timeout_s, out, max_out, &n);
    *n_out = n;
    return rc;
}

pb_status pb_engine_query(pb_engine *e, int32_t *n_pending, int32_t *n_active, int64_t *replays) {
    set_error("");
    if (!e) {
        set_error("pb_engine_query: NULL engine");
        return PB_ERR_ARG;
    }
    int p = 0, a = 0;
    long long r = 0;
    pb_status rc = engine_query(e, &p, &a, &r);
    if (n_pending) *n_pending = p;
    if (n_active) *n_active = a;
    if (replays) *replays = r;
    return rc;
}

pb_status pb_engine_destroy(pb_engine *e) {
    set_error("");
    if (!e) return PB_OK;
    return engine_destroy(e);
}

pb_status pb_profile_kernels(pb_system *s, int32_t precision, int32_t which, int32_t reps,
                             void *stream) {
    set_error("");
    if (!s || (precision != PB_FP64 && precision != PB_MIXED) || which < 0 || which > 2 ||
        reps < 0) {
        set_error("pb_profile_kernels: bad argument");
        return PB_ERR_ARG;
    }
    if ((precision == PB_MIXED && !s->z32) || (precision == PB_FP64 && !s->z64)) {
        set_error("pb_profile_kernels needs a prior pb_solve in that precision");
        return PB_ERR_STATE;
    }
    DeviceGuard dg(s->g->device);
    if (s->g->is_oct) return oct_profile(s, precision, which, reps, (cudaStream_t)stream);
    return profile_kernels(s, precision, which, reps, (cudaStream_t)stream);
}

int64_t pb_kernel_launches(void) { return g_launches.load(); }

pb_status pb_set_tuning(pb_system *s, int32_t precision, int32_t variant, int32_t z_chunk) {
    set_error("");
    if (!s || (precision != PB_FP64 && precision != PB_MIXED)) {
        set_error("pb_set_tuning: bad argument");
        return PB_ERR_ARG;
    }
    if (s->g->is_oct) {
        set_error("pb_set_tuning: octree kernels have no tuning parameters");
        return PB_ERR_UNIMPL;
    }
    return set_tuning(s, precision, variant, z_chunk);
}

pb_status pb_solve_split(pb_system *s, int32_t ranks, const pb_solve_opts *opts, void *stream,
                         pb_solve_stats *stats) {
    set_error("");
    if (!s) {
        set_error("pb_solve_split: NULL system");
        return PB_ERR_ARG;
    }
    pb_status rc = check_opts(opts);
    if (rc != PB_OK) return rc;
    if (opts->precision != PB_MIXED) {
        set_error("pb_solve_split: the split solve runs the mixed-precision solver");
        return PB_ERR_ARG;
    }
    if (s->g->is_oct) {
        set_error("pb_solve_split: octree systems are solved by pb_solve");
        return PB_ERR_UNIMPL;
    }
    DeviceGuard dg(s->g->device);
    rc = solve_split(s, ranks, opts, (cudaStream_t)stream, stats);
    if (rc == PB_ERR_NOCONV) set_error("solver stopped before reaching rtol");
    if (rc == PB_ERR_TIMEOUT && !g_err[0]) set_error("solver exceeded its time budget");
    return rc;
}

pb_status pb_set_wait_limit(int64_t polls) {
    set_error("");
    return set_wait_limit((long long)polls);
}

}  // extern "C"

