// Energy terms of Sec. 3.3 from the solved potential.
//
// For every flux edge (endpoints in different media) with inside endpoint
// "in" and outward unit direction n_e:
//   F_e   = W_e (phi_in - phi_out)        flux of D^eff through the dual face
//                                          (Eq. Dnvh_approx, times 4 pi l_B)
//   q_e   = (1/eps_s - 1/eps_m) F_e / (4 pi l_B), placed at r_e (Sec. 3.3.1)
//   phi_e = phi_in + (alpha/eps_m)(phi_out - phi_in) / (alpha/eps_m + (1-alpha)/eps_s)
//                                          (Eq. phi0)
// E_pol      = 1/2 (1/eps_s - 1/eps_m) sum_e F_e Phi_e / (4 pi)
// E_ion_flux = -1/2 (1/eps_s) sum_e F_e Phi_e / (4 pi)    (Eq. energy_ion, 2nd)
// E_ion_surf = 1/2 sum_e phi_e h^2 Psi_e / (4 pi)          (Eq. energy_ion, 1st,
//                                                            staircase faces)
// E_ion_mc   = 1/2 sum_e T_e phi_e Psi^n_e / (4 pi)        (Eq. energy_ion, 1st,
//              on the surface re-triangulated by marching cubes, Sec. 3.3.2:
//              T_e the vertex weight, Psi^n_e along the analytic normal)
// E_coul     = (l_B/eps_m) 1/2 sum_i q_i sum_{j!=i} q_j / r_ij
// All sums FP64, reduced in a fixed order.
#include <math.h>

#include <algorithm>

#include "pb_internal.h"

namespace pbg {

namespace {

constexpr int EN_THREADS = 256;

__device__ __forceinline__ double bsum(double v, double *sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sred[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < EN_THREADS / 32; ++q) t += sred[q];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(EN_THREADS)
k_energy(const long long *__restrict__ ids, const double *__restrict__ alpha,
         const int8_t *__restrict__ sign, long long ncross, const double *__restrict__ Wx,
         const double *__restrict__ Wy, const double *__restrict__ Wz,
         const double *__restrict__ phi, const double *__restrict__ Phi,
         const double *__restrict__ Psi, const double *__restrict__ Tw,
         const double *__restrict__ PsiN, GridGeo g, double eps_in, double eps_out, double lB,
         double *partials, EnergyAcc *acc) {
    __shared__ double sred[EN_THREADS / 32];
    __shared__ int s_last;
    double S = 0.0, I = 0.0, F = 0.0, Im = 0.0;
    for (long long s = blockIdx.x * (long long)EN_THREADS + threadIdx.x; s < ncross;
         s += (long long)gridDim.x * EN_THREADS) {
        int sg = sign[s];
        if (sg == 0) continue;
        long long e = ids[s];
        int d = (int)(e / g.N);
        long long a = e - (long long)d * g.N;
        long long st = d == 0 ? 1 : (d == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
        long long b = a + st;
        const double *W = d == 0 ? Wx : (d == 1 ? Wy : Wz);
        long long in = sg > 0 ? a : b, out = sg > 0 ? b : a;
        double pin = phi[in], pout = phi[out];
        double Fe = W[a] * (pin - pout);
        double al = alpha[s];
        double phip = pin + (al / eps_in) * (pout - pin) / (al / eps_in + (1.0 - al) / eps_out);
        S += Fe * Phi[s];
        I += phip * (g.h * g.h) * Psi[s];
        F += Fe;
        if (Tw) Im += Tw[s] * phip * PsiN[s];
    }
    double bS = bsum(S, sred), bI = bsum(I, sred), bF = bsum(F, sred), bM = bsum(Im, sred);
    int nb = gridDim.x;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bS;
        partials[nb + blockIdx.x] = bI;
        partials[2 * nb + blockIdx.x] = bF;
        partials[3 * nb + blockIdx.x] = bM;
        __threadfence();
        unsigned t = atomicAdd(&acc->counter, 1u);
        s_last = (t == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int q = threadIdx.x; q < nb; q += EN_THREADS) {
        a0 += __ldcg(partials + q);
        a1 += __ldcg(partials + nb + q);
        a2 += __ldcg(partials + 2 * nb + q);
        a3 += __ldcg(partials + 3 * nb + q);
    }
    double tS = bsum(a0, sred), tI = bsum(a1, sred), tF = bsum(a2, sred), tM = bsum(a3, sred);
    if (threadIdx.x == 0) {
        const double fourpi = 4.0 * M_PI;
        acc->S = tS;
        acc->I = tI;
        acc->F = tF;
        acc->Imc = tM;
        pb_energy_terms o{};
        o.e_coul = (lB / eps_in) * 0.5 * acc->ecoul_sum;
        o.e_pol = 0.5 * (1.0 / eps_out - 1.0 / eps_in) * tS / fourpi;
        o.e_ion_flux = -0.5 * (1.0 / eps_out) * tS / fourpi;
        o.e_ion_surf = 0.5 * tI / fourpi;
        o.e_total = o.e_coul + o.e_pol + o.e_ion_surf + o.e_ion_flux;
        o.flux_charge = tF / (fourpi * lB);
        o.e_ion_mc = 0.5 * tM / fourpi;
        acc->out = o;
        acc->counter = 0;
    }
}

}  // namespace

pb_status energy(pb_system *sys, cudaStream_t s, pb_energy_terms *out) {
    pb_grid *g = sys->g;
    int nb = (int)std::min<long long>(cdiv(g->ncross > 0 ? g->ncross : 1, EN_THREADS),
                                      (long long)num_sms() * 8);
    double *partials = (double *)dalloc(sizeof(double) * 4 * nb, s);
    if (!partials) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(&sys->eacc->counter, 0, sizeof(unsigned), s));
    k_energy<<<nb, EN_THREADS, 0, s>>>(g->cid, g->calpha, g->csign, g->ncross, sys->W[0], sys->W[1],
                                       sys->W[2], sys->phi, sys->Phi, sys->Psi,
                                       g->mc_w, sys->PsiN, g->geo,
                                       sys->p.eps_in, sys->p.eps_out, sys->lB, partials, sys->eacc);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(sys->h_energy, &sys->eacc->out, sizeof(pb_energy_terms),
                                cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(partials, s);
    *out = *sys->h_energy;
    return PB_OK;
}

}  // namespace pbg
