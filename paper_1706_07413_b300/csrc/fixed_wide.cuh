// fixed_wide.cuh -- one instance of the fixed-metric scheme evolved by the whole GPU.
//
// The paper's Table II case (Sec. IV): A = 1 and delta = 0 held fixed, so that Eqs. (eq:phi),
// (eq:pi) are the linear wave equation on AdS4, stepped with the Shu-Osher SSP-RK3 method.  The
// persistent kernels of evolve_ea.cuh give one instance at most one 16-CTA cluster (16 of the
// SMs); here a single instance is spread over a cooperative launch of ceil(N / kWideNT) CTAs, one
// grid node per thread, and the CTAs meet at one grid-wide barrier per Runge-Kutta stage:
//   stage s: barrier (the stage slice y_s and u_s = tan^2 x Phi_s are complete everywhere);
//            each CTA stages its node block with a 3-node halo (parity ghosts at both ends) from
//            L2 into shared memory, forms Phi-dot, Pi-dot on its nodes and writes
//            y_{s+1} = a_s y_n + b_s (y_s + dt L(y_s)) with u_{s+1} for its nodes.
// Readings as in the rest of the solver: Phi-dot = D(Pi) and Pi-dot = tan^{-2} x D(tan^2 x Phi)
// with the 4th-order difference D and Kreiss-Oliger dissipation sigma/(64 h) Delta^6 on every
// non-boundary row; Pi-dot(0) = 3 D(Phi)(0) plus dissipation; Phi(0), Phi(pi/2), Pi(pi/2) held;
// u(pi/2) by the even extrapolation (4 u_{N-2} - u_{N-3}) / 3.  Stage data written by other SMs
// are read with ld.global.cg (L2), never through a possibly stale L1 line.  The barrier's wait
// has an iteration limit: when it runs out the kernel records it and returns, and the instance is
// reported TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "evolve.cuh"

namespace adscl {

constexpr int kWideNT = 512;   // threads (= grid nodes) per CTA

struct WideArgs {
    InstDesc d;               // the instance's coefficients (h, dt, dissipation)
    const double *T;          // tan^2 x (0 at pi/2)
    const double *iT12;       // 1 / (12 h tan^2 x) (0 at both ends)
    const double *wsim;       // weights of the slice mass: (h/3) Simpson weight tan^2 x
    double *Phi, *Pi;         // the slice y_n (updated in place)
    double *Y1P, *Y1Q, *Y2P, *Y2Q;   // stage slices y_1, y_2
    double *U0, *U1;          // u = tan^2 x Phi of the stage slice read / written (alternating)
    InstState *st;            // the instance's state record (step, diagnostics, status)
    long long n_end;          // evolve until the step index reaches n_end
    unsigned *bar;            // grid barrier: [0] arrivals, [1] generation
    int *flag;                // [0] a non-finite value was written, [1] a barrier wait ran out
    double *part;             // per-CTA partial sums of the slice mass
    long long max_spin;       // iteration limit of a barrier wait
};

// gpu-scope acquire load, acquire-release atomic add and release add (PTX memory model)
__device__ __forceinline__ unsigned wide_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned wide_atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void wide_red_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch: every CTA's writes before it are visible to every
// CTA after it.  The CTA barrier orders the CTA's writes before thread 0's arrival, a release at
// gpu scope (cumulative); the last arrival resets the count and releases the next generation,
// which the others acquire.  Returns false if this CTA's wait ran out (flag[1] is then set).
__device__ __forceinline__ bool wide_barrier(unsigned *bar, int *flag, long long max_spin)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = wide_ld_acquire(bar + 1);
        int ok = 1;
        if (wide_atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);          // ordered before the release below
            wide_red_release(bar + 1, 1u);
        } else {
            long long it = 0;
            while (wide_ld_acquire(bar + 1) == g) {
                if (++it > max_spin) {
                    atomicExch(flag + 1, 1);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok && (*(volatile int *)(flag + 1) == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// value of a node array at index j in [-3, N+2] read from L2, with the parity ghosts
// u_{-k} = p0 u_k and u_{N-1+k} = p1 u_{N-1-k}
__device__ __forceinline__ double wide_ghost(const double *u, int N, int j, double p0, double p1)
{
    if (j < 0) return p0 * __ldcg(u - j);
    if (j > N - 1) return p1 * __ldcg(u + 2 * (N - 1) - j);
    return __ldcg(u + j);
}

__global__ void __launch_bounds__(kWideNT, 1) fixed_wide_kernel(WideArgs a)
{
    constexpr int NT = kWideNT;
    __shared__ double tP[NT + 6], tQ[NT + 6], tU[NT + 4];   // stage slice and u, with halos
    __shared__ double s_red[NT / 32];
    const InstDesc &d = a.d;
    const int N = d.N, tid = threadIdx.x;
    const int i0 = blockIdx.x * NT, i = i0 + tid;
    const bool act = i < N;
    const double aco[3] = {0.0, 0.75, 1.0 / 3.0}, bco[3] = {1.0, 0.25, 2.0 / 3.0};

    const long long step0 = a.st->step;
    const bool running = a.st->status == kRunning;
    const long long nsteps = (running && a.n_end > step0) ? a.n_end - step0 : 0;

    // u of the slice y_n
    int cu = 0;   // the u buffer of the slice being read: 0 -> U0, 1 -> U1
    if (act) a.U0[i] = (i < N - 1) ? mul_f(__ldg(a.T + i), a.Phi[i]) : 0.0;

    long long done = 0;
    bool ok = true;
    for (long long n = 0; n < nsteps && ok; ++n) {
        for (int s = 0; s < 3; ++s) {
            if (!(ok = wide_barrier(a.bar, a.flag, a.max_spin))) break;
            if (s == 0 && __ldcg(a.flag) != 0) { ok = false; break; }   // the last slice is not finite
            const double *yP = (s == 0) ? a.Phi : (s == 1) ? a.Y1P : a.Y2P;
            const double *yQ = (s == 0) ? a.Pi : (s == 1) ? a.Y1Q : a.Y2Q;
            const double *uS = cu ? a.U1 : a.U0;
            double *oP = (s == 0) ? a.Y1P : (s == 1) ? a.Y2P : a.Phi;
            double *oQ = (s == 0) ? a.Y1Q : (s == 1) ? a.Y2Q : a.Pi;
            double *uO = cu ? a.U0 : a.U1;
            // the block's stage slice with its halo: Phi odd / even, Pi even / odd, u odd / even
            // about x = 0 / pi/2; u(pi/2) by the even extrapolation
            for (int k = tid; k < NT + 6; k += NT) {
                const int j = i0 - 3 + k;
                if (j <= N + 2) {
                    tP[k] = wide_ghost(yP, N, j, -1.0, 1.0);
                    tQ[k] = wide_ghost(yQ, N, j, 1.0, -1.0);
                }
            }
            for (int k = tid; k < NT + 4; k += NT) {
                const int j = i0 - 2 + k;
                if (j <= N + 1) {
                    tU[k] = (j == N - 1) ? (4.0 * __ldcg(uS + N - 2) - __ldcg(uS + N - 3)) * (1.0 / 3.0)
                                         : wide_ghost(uS, N, j, -1.0, 1.0);
                }
            }
            __syncthreads();
            if (act) {
                const double *p = tP + tid + 3, *q = tQ + tid + 3, *u = tU + tid + 2;
                const double kop = fma(-20.0, p[0], fma(15.0, add_f(p[-1], p[1]), fma(-6.0, add_f(p[-2], p[2]), add_f(p[-3], p[3]))));
                const double koq = fma(-20.0, q[0], fma(15.0, add_f(q[-1], q[1]), fma(-6.0, add_f(q[-2], q[2]), add_f(q[-3], q[3]))));
                double dP = 0.0, dQ = 0.0;
                if (i == 0) {
                    dQ = fma(d.c3, fma(16.0, p[1], -2.0 * p[2]), mul_f(d.cko, koq));
                } else if (i < N - 1) {
                    const double Df = fma(8.0, add_f(q[1], -q[-1]), add_f(q[-2], -q[2]));
                    const double Du = fma(8.0, add_f(u[1], -u[-1]), add_f(u[-2], -u[2]));
                    dP = fma(d.c12, Df, mul_f(d.cko, kop));
                    dQ = fma(__ldg(a.iT12 + i), Du, mul_f(d.cko, koq));
                }
                // y_{s+1} = a_s y_n + b_s (y_s + dt L(y_s))
                const double sP = fma(d.dt, dP, p[0]), sQ = fma(d.dt, dQ, q[0]);
                double nP = (s == 0) ? sP : fma(aco[s], a.Phi[i], mul_f(bco[s], sP));
                double nQ = (s == 0) ? sQ : fma(aco[s], a.Pi[i], mul_f(bco[s], sQ));
                oP[i] = nP;
                oQ[i] = nQ;
                uO[i] = (i < N - 1) ? mul_f(__ldg(a.T + i), nP) : 0.0;
                if (s == 2 && !(isfinite(nP) && isfinite(nQ))) atomicExch(a.flag, 1);
            }
            cu ^= 1;
        }
        if (ok) done = n + 1;
    }
    // the slice mass: per-CTA partial sums, then CTA 0 adds them in CTA order
    const bool synced = wide_barrier(a.bar, a.flag, a.max_spin);
    double ms = 0.0;
    if (act) {
        const double ph = __ldcg(a.Phi + i), pi = __ldcg(a.Pi + i);
        ms = mul_f(__ldg(a.wsim + i), fma(ph, ph, mul_f(pi, pi)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ms += __shfl_xor_sync(0xffffffffu, ms, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = ms;
    __syncthreads();
    if (tid == 0) {
        double b = s_red[0];
        for (int w = 1; w < NT / 32; ++w) b += s_red[w];
        a.part[blockIdx.x] = b;
    }
    const bool synced2 = wide_barrier(a.bar, a.flag, a.max_spin);
    if (blockIdx.x == 0 && tid == 0) {
        double m = __ldcg(a.part);
        for (unsigned c = 1; c < gridDim.x; ++c) m += __ldcg(a.part + c);
        InstState *S = a.st;
        S->step = step0 + done;
        if (nsteps > 0) {
            S->mass = m;
            S->minA = 1.0;
            S->delta0 = 0.0;
        }
        const bool timeout = !synced || !synced2 || __ldcg(a.flag + 1) != 0;
        if (timeout) S->status = kTimeout;
        else if (__ldcg(a.flag) != 0 || !isfinite(m)) S->status = kNonfinite;
    }
}

}  // namespace adscl
