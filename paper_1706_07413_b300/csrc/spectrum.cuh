// spectrum.cuh -- AdS4 normal modes on the grid: mode-sum initial data and the mode-energy
// spectrum E_j = Pi_j^2 + Phi_j^2 / omega_j^2 of arXiv:1706.07413, Sec. II (the solution at
// any time is projected onto the normal modes).
//
// Normal modes (the paper gives no formula; standard for a massless scalar on AdS4):
//   e_j(x) = cos^3 x q_j(cos 2x),  omega_j = 3 + 2j,  int_0^{pi/2} e_i e_j tan^2 x dx = delta_ij,
// with q_j = 4 p_j and p_j the orthonormal polynomials of the weight (1-y)^{1/2} (1+y)^{3/2} on
// [-1, 1], generated on the host by their three-term (Jacobi-matrix) recurrence
//   y p_n = a_{n+1} p_{n+1} + b_n p_n + a_n p_{n-1},
//   a_n = sqrt(n (n+2)) / (2 (n+1)),  b_n = 1 / (2 (n+1) (n+2)),  p_0 = sqrt(2/pi),
// and e_j' from the differentiated recurrence.  Projections (the trapezoid rule on the grid;
// the integrand vanishes at both ends):
//   Pi_j = h sum_i tan^2 x_i sqrt(A_i) Pi_i e_j(x_i),  Phi_j = h sum_i tan^2 x_i sqrt(A_i) Phi_i e_j'(x_i).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "evolve.cuh"

namespace adscl {

constexpr int kMaxModes = 64;

struct EigTab {
    const double *e;   // kMaxModes x N: e_j(x_i)
    const double *de;  // kMaxModes x N: e_j'(x_i)
};

// Pi(x,0) = sum_{j<K} a_j e_j(x), Phi(x,0) = 0 for every instance (one CTA per instance)
__global__ void synth_kernel(const InstDesc *desc, const EigTab *eig, const double *a, int K,
                             double *Phi, double *Pi)
{
    const int b = blockIdx.x;
    const InstDesc d = desc[b];
    const EigTab t = eig[d.geo];
    const double *ab = a + (size_t)b * K;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s = fma(__ldg(ab + j), __ldg(t.e + (size_t)j * d.N + i), s);
        Pi[d.off + i] = (i == d.N - 1) ? 0.0 : s;
        Phi[d.off + i] = 0.0;
    }
}

// projection weights w_i = h tan^2 x_i sqrt(A_i) on interior nodes, times Pi and Phi
// (one CTA per instance); u = w Pi, v = w Phi, packed like the fields
__global__ void spectrum_weights_kernel(const InstDesc *desc, const GeoTab *geo, const double *Phi,
                                        const double *Pi, const double *A, double *u, double *v)
{
    const int b = blockIdx.x;
    const InstDesc d = desc[b];
    const GeoTab g = geo[d.geo];
    const double h = 1.0 / (12.0 * d.c12);
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        double w = 0.0;
        if (i > 0 && i < d.N - 1) w = h * __ldg(g.T + i) * sqrt(A[d.off + i]);
        u[d.off + i] = w * Pi[d.off + i];
        v[d.off + i] = w * Phi[d.off + i];
    }
}

// FP64 projection: E[b*J + j] (one CTA per instance, one warp per mode at a time)
__global__ void spectrum_fp64_kernel(const InstDesc *desc, const EigTab *eig, const double *u,
                                     const double *v, int J, double *E)
{
    const int b = blockIdx.x;
    const InstDesc d = desc[b];
    const EigTab t = eig[d.geo];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double *ub = u + d.off, *vb = v + d.off;
    for (int j = warp; j < J; j += nw) {
        const double *ej = t.e + (size_t)j * d.N, *dj = t.de + (size_t)j * d.N;
        double sp = 0.0, sf = 0.0;
        for (int i = lane; i < d.N; i += 32) {
            sp = fma(__ldg(ub + i), __ldg(ej + i), sp);
            sf = fma(__ldg(vb + i), __ldg(dj + i), sf);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sf += __shfl_xor_sync(0xffffffffu, sf, o);
        }
        if (lane == 0) {
            const double w = 3.0 + 2.0 * j;
            E[(size_t)b * J + j] = fma(sp, sp, sf * sf / (w * w));
        }
    }
}

// Two of the three quantities conserved by the two-time-framework (TTF) equations, from the
// mode energies of each instance (one thread per instance): the total energy E = sum_j E_j and
// the particle number N = sum_j E_j / omega_j (E_j / omega_j: the quanta in mode j), with the
// temperature T = E / N (Sec. II quotes T for its quasi-periodic data).  Summed in order of j.
// out[3b + 0..2] = E, N, T.  The third TTF quantity needs interaction coefficients the paper
// does not give.
__global__ void ttf_kernel(const double *E, int B, int J, double *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double *e = E + (size_t)b * J;
    double et = 0.0, nt = 0.0;
    for (int j = 0; j < J; ++j) {
        const double v = e[j];
        et += v;
        nt += v / (3.0 + 2.0 * j);
    }
    out[3 * b] = et;
    out[3 * b + 1] = nt;
    out[3 * b + 2] = et / nt;
}

}  // namespace adscl
