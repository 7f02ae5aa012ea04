// Internal declarations shared by the CUDA translation units of libpbgpu.
// Nothing here is part of the public C ABI (include/pb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pb.h"

namespace pbg {

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
void note_launch(long long n);
#define PB_CUDA_TRY(expr)                                                         \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::pbg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                 \
            return PB_ERR_CUDA;                                                   \
        }                                                                         \
    } while (0)
#define PB_LAUNCH_CHECK()          \
    do {                           \
        ::pbg::note_launch(1);     \
        PB_CUDA_TRY(cudaGetLastError()); \
    } while (0)

// ------------------------------------------------------------- allocator --
void *dalloc(size_t bytes, cudaStream_t s);   // nullptr on failure
void dfree(void *p, cudaStream_t s);

// Device-side error flags written by kernels (bit mask).
enum : uint32_t {
    ERRF_ATOM_VALUE = 1u,      // NaN/Inf coordinate or non-positive radius
    ERRF_CHARGE_CELL = 2u,     // a charge's trilinear cell touches the boundary
    ERRF_TOO_MANY_BALLS = 4u,  // more than MAX_EDGE_BALLS balls meet one listed edge
    ERRF_CELL_OVERFLOW = 8u,   // atom cell list inconsistent
};
constexpr int MAX_EDGE_BALLS = 48;

// Geometry and build summary computed on the device and read back once.
struct BuildInfo {
    double lo[3], hi[3];  // bounding box of the atom balls
    double origin[3], h;  // grid placement
    double rmax;          // largest radius
    uint32_t err;         // ERRF_* bits
    uint32_t pad;
    unsigned long long ncross, nflux, ninside;
};

// Atom cell list used by the crossing-edge pass and the charge deposit.
struct CellList {
    double lo[3];     // corner of cell (0,0,0)
    double cs;        // cell side
    int dim[3];
    int ncell;
    int *start;       // [ncell + 1]
    int *atom;        // [na] atom ids grouped by cell
};

// Grid geometry passed by value to kernels.
struct GridGeo {
    int nx, ny, nz;
    long long N;          // nx*ny*nz (canonical node count)
    double o[3];
    double h;
};

// Padded FP32/FP64 solver layout: rows padded to a multiple of 4 elements.
struct PadGeo {
    int nx, ny, nz;
    int sx;               // padded row length
    long long sxy;        // sx * ny
    long long Np;         // sx * ny * nz
    long long N;          // canonical nx*ny*nz
};

// Octree brick grid (device arrays and scalars, passed by value to kernels).
// Positions are integers in units of the finest spacing ("node units");
// brick b owns the 8^3 low-corner nodes of its cells, slot 512 b + (8k+j)8+i.
struct OctDev {
    double o[3];
    double hf;            // finest spacing
    int Lmax, n0, nf, NL; // levels - 1, coarse bricks per axis, finest bricks per axis, side
    long long nb, N;      // bricks, node slots (512 nb)
    uint8_t *lev;         // [nf^3] leaf level of each finest-brick cell, (cz*nf+cy)*nf+cx
    int *bmap;            // [nf^3] leaf brick covering each finest-brick cell
    int4 *blow;           // [nb] low corner (node units) and level
    int *bnbr;            // [6 nb] same-level face neighbour (-x,+x,-y,+y,-z,+z); -1 other
                          // level, -2 outside the domain
    uint8_t *okind;       // [N] 0 pure row, 1 boundary, 2 hanging, 3 level-transition row
};

// Level-transition rows of an octree system: explicit CSR of P^T K P.
struct OctSys {
    long long ntr, nnz;
    long long nunk;       // unknowns (pure and level-transition rows)
    int *tr_slot;         // [ntr] slot of each row (increasing)
    int *tr_row;          // [N] row of each slot, -1 if none
    long long *tr_ptr;    // [ntr + 1]
    int *tr_col;          // [nnz] column slots, increasing within a row
    double *tr_val;       // [nnz]
    float *tr_val32;      // [nnz]
    double *tr_diag;      // [ntr]
    double *tpart;        // [4] totals of the transition kernels (sigma, rho, rr)
    double *partials;     // per-block partials of the transition kernels
    unsigned int *tcount; // last-block counter of the transition kernels
    int npart;
};

}  // namespace pbg

struct pb_grid {
    int device;
    cudaStream_t stream;  // creation stream; memory is released on it
    pbg::GridGeo geo;
    long long na;
    double *atoms;        // SoA: x[na], y[na], z[na], R[na], q[na]
    uint8_t *inside;      // [N] 1 = solute
    pbg::CellList cells;
    long long ncross, nflux, ninside;
    long long *cid;       // [ncross] edge ids, increasing
    double *calpha;       // [ncross]
    double *crp;          // [3*ncross] AoS
    int8_t *csign;        // [ncross]
    int *rowstart;        // [3*ny*nz + 1] first list entry of each edge row
    pbg::BuildInfo *d_info;
    double center[3];     // shift used by the FP32 N-body kernels
    int is_oct;           // octree grid: geo is the flat slot layout (nx = N)
    pbg::OctDev ot;
    pbg::GridGeo vgeo;    // octree: the uniform lattice at the finest spacing
    long long *cslot_b;   // octree: slot of the +d end of each listed edge
    double *mc_w;         // [ncross] re-triangulated surface: vertex weight (sum of T_j/3)
    double *mc_n;         // [3 ncross] analytic outward unit normal at each crossing point
};

namespace pbg {

// Device scalars of one PCG solve.
struct CgState {
    double rho;      // r.z of the current iterate
    double alpha, beta;
    double rr;       // ||r||^2 of the current iterate
    double rr_stop;  // stop when rr <= rr_stop
    double rr0;
    double sigma;
    double res64;    // ||f - A phi||^2 from the FP64 residual pass
    double rz64;     // r.(r/diag) from the FP64 residual pass
    int iter;        // iterations done
    int max_iter;
    int done;        // 1 = converged or stopped
    int status;      // 0 ok, 1 breakdown, 2 max_iter
    unsigned int counter;  // last-block counter of the reductions
    int profile;     // 1 = timing run: never stop
    int cur;         // FP32 TMA kernels: which of pa/pb holds p_old (flips per iteration)
    int split;       // 1: one slab of a split solve (the launch stores its totals in
                     // part0/part1; the CG update runs after the rank-ordered sum)
    double part0, part1;
};

struct EnergyAcc {
    double S, I, F;  // sum F*Phi, sum phi(rp) h^2 Psi, sum F
    double Imc;      // sum W phi(rp) Psi_n over the re-triangulated surface
    double ecoul_sum;
    pb_energy_terms out;
    unsigned int counter;
    unsigned int pad;
};

}  // namespace pbg

struct pb_system {
    pb_grid *g;
    cudaStream_t stream;
    pb_params p;
    double lB, kD, kap_s;
    double *W[3];       // canonical FP64 edge weights
    double *diag;       // canonical FP64 diagonal (0 on boundary)
    double *rhs;        // canonical f
    double *bc;         // canonical boundary values (0 inside)
    double *phi;        // canonical solution incl. boundary values
    pbg::PadGeo pad;
    uint8_t *code;      // padded: bit0 solute, bit1..3 +x/+y/+z edge listed
    float *w32[3];      // padded FP32 edge weights (read only where listed)
    // FP32 mixed solver workspace (padded layout)
    float *z32, *pa32, *pb32, *d32;
    // FP64 plain solver workspace (padded layout)
    double *z64, *pa64, *pb64, *x64;
    double *r64, *q64;  // plain FP64 solver: residual and q = A p (padded)
    double *op64[5];    // plain FP64 solver: padded +x/+y/+z weights, diagonal, 1/diagonal
    double *partials;   // reduction partials
    int npartials;
    pbg::CgState *st;
    pbg::CgState *h_st; // pinned host mirror
    double *Phi, *Psi;  // [ncross]
    double *PsiN;       // [ncross] Psi along the grid's analytic normals (mc_n)
    pbg::EnergyAcc *eacc;
    pb_energy_terms *h_energy;  // pinned
    int solved, have_surface, have_pairs;
    double fnorm2;
    void *tma;          // tensor maps of the FP32 stencil kernels (host object)
    unsigned int *queue;  // work counters of the TMA stencil kernels (device)
    pbg::OctSys *os;    // octree systems: level-transition rows
};

namespace pbg {

// ---------------------------------------------------------------- grid.cu --
pb_status grid_build(pb_grid *g, const pb_grid_spec *spec, cudaStream_t s);

// ----------------------------------------------------------- assemble.cu --
pb_status assemble(pb_system *sys, cudaStream_t s);
pb_status deposit_rhs(pb_system *sys, cudaStream_t s);
pb_status fill_kappa(const pb_system *sys, double *dst, cudaStream_t s);

// -------------------------------------------------------------- nbody.cu --
pb_status nbody_boundary(pb_system *sys, cudaStream_t s);
pb_status nbody_surface(pb_system *sys, cudaStream_t s);
pb_status nbody_pairs(pb_system *sys, cudaStream_t s);

// ------------------------------------------------------------ surface.cu --
pb_status mc_surface(pb_grid *g, cudaStream_t s);

// -------------------------------------------------------------- solve.cu --
pb_status solve(pb_system *sys, const pb_solve_opts *o, cudaStream_t s, pb_solve_stats *st);
pb_status apply_op(pb_system *sys, int precision, const void *x, void *y, cudaStream_t s);
pb_status ensure_solver_ws(pb_system *sys, int precision, cudaStream_t s);
pb_status profile_kernels(pb_system *sys, int precision, int which, int reps, cudaStream_t s);
void free_tma_state(pb_system *sys);
pb_status set_tuning(pb_system *sys, int precision, int variant, int kc);
pb_status set_wait_limit(long long polls);
pb_status solve_batch(pb_system *const *systems, int n, const pb_solve_opts *o, cudaStream_t s,
                      pb_solve_stats *stats);
pb_status solve_split(pb_system *sys, int ranks, const pb_solve_opts *o, cudaStream_t s,
                      pb_solve_stats *stats);
pb_status engine_create(int device, int capacity, const pb_solve_opts *o, pb_engine **out);
pb_status engine_submit(pb_engine *e, pb_system *sys, cudaStream_t s, long long *ticket);
pb_status engine_wait(pb_engine *e, double timeout_s, pb_engine_result *out, int max_out, int *n_out);
pb_status engine_query(pb_engine *e, int *n_pending, int *n_active, long long *replays);
pb_status engine_destroy(pb_engine *e);

// ------------------------------------------------------------- octree.cu --
pb_status oct_build(pb_grid *g, const pb_grid_spec *spec, cudaStream_t s);
void oct_grid_free(pb_grid *g, cudaStream_t s);
pb_status oct_assemble(pb_system *sys, cudaStream_t s);
pb_status oct_boundary_rhs(pb_system *sys, cudaStream_t s);
void oct_system_free(pb_system *sys, cudaStream_t s);
pb_status oct_solve(pb_system *sys, const pb_solve_opts *o, cudaStream_t s, pb_solve_stats *st);
pb_status oct_apply(pb_system *sys, int precision, const void *x, void *y, cudaStream_t s);
pb_status oct_energy(pb_system *sys, cudaStream_t s, pb_energy_terms *out);
pb_status oct_fill_kappa(const pb_system *sys, double *dst, cudaStream_t s);
pb_status oct_profile(pb_system *sys, int precision, int which, int reps, cudaStream_t s);
pb_status oct_engine_prepare(pb_system *sys, cudaStream_t s);
pb_status oct_engine_residual(pb_system *sys, cudaStream_t s);
pb_status oct_engine_promote(pb_system *sys, cudaStream_t s);
pb_status oct_engine_iterations(pb_system *sys, int n, cudaStream_t s);

// ------------------------------------------------------------- energy.cu --
pb_status energy(pb_system *sys, cudaStream_t s, pb_energy_terms *out);

// helpers
inline unsigned int cdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }
inline int num_sms() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
    }
    return v;
}

}  // namespace pbg
