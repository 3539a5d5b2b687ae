// fixed_wide.cuh -- one instance of the fixed-metric scheme evolved by the whole GPU.
//
// The paper's Table II case (Sec. IV): A = 1 and delta = 0 held fixed, so that Eqs. (eq:phi),
// (eq:pi) are the linear wave equation on AdS4, stepped with the Shu-Osher SSP-RK3 method.  The
// persistent kernels of evolve_ea.cuh give one instance at most one 16-CTA cluster (16 of the
// SMs); here a single instance is spread over a cooperative launch of ceil(N / kWideNodes) CTAs
// of kWideNT threads, and the CTAs meet once per step:
//   step n: grid barrier (every CTA has written its nodes of y_n); each CTA copies from L2 the
//           slice on its kWideNodes nodes and kWideHalo = 9 nodes on each side (three stages of the
//           3-node stencil reach), with the parity ghosts at both ends, into shared memory; it then
//           forms the three stages on shrinking ranges (its nodes and 6, 3, 0 nodes on each side:
//           512, 506, 500 nodes, so that the 16 warps stay full) with u = tan^2 x Phi computed
//           locally, and writes y_{n+1} on its own nodes to the other of two global slices (the
//           neighbours may still be reading the current one) before arriving at the next barrier.
// Readings as in the rest of the solver: Phi-dot = D(Pi) and Pi-dot = tan^{-2} x D(tan^2 x Phi)
// with the 4th-order difference D and Kreiss-Oliger dissipation sigma/(64 h) Delta^6 on every
// non-boundary row; Pi-dot(0) = 3 D(Phi)(0) plus dissipation; Phi(0), Phi(pi/2), Pi(pi/2) held;
// u(pi/2) by the even extrapolation (4 u_{N-2} - u_{N-3}) / 3.  The slice written by other SMs is
// read with ld.global.cg (L2), never through a possibly stale L1 line.  The barrier's wait has an
// iteration limit: when it runs out the kernel records it and returns, and the instance is
// reported TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "evolve.cuh"

namespace adscl {

constexpr int kWideNT = 512;     // threads per CTA
constexpr int kWideNodes = 500;  // grid nodes owned by a CTA
constexpr int kWideHalo = 9;     // nodes copied on each side: 3 stages x the 3-node stencil reach

struct WideArgs {
    InstDesc d;               // the instance's coefficients (h, dt, dissipation)
    const double *T;          // tan^2 x (0 at pi/2)
    const double *iT12;       // 1 / (12 h tan^2 x) (0 at both ends)
    const double *wsim;       // weights of the slice mass: (h/3) Simpson weight tan^2 x
    double *Phi, *Pi;         // the slice (in and out)
    double *BP, *BQ;          // the other global slice (the steps alternate between the two)
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

// Grid-wide barrier of a cooperative launch, split into an arrival and a wait so that a CTA can
// work between them.  Thread 0 arrives after a CTA barrier (which orders the CTA's writes before
// its gpu-scope release); the last arrival resets the count and releases the next generation,
// which the waiting CTAs acquire.  Every arrival is waited for before the CTA's next arrival.
// wide_arrive returns the generation to wait past; wide_wait returns false if its wait ran out
// (flag[1] is then set).
__device__ __forceinline__ unsigned wide_arrive(unsigned *bar)
{
    const unsigned g = wide_ld_acquire(bar + 1);
    if (wide_atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
        atomicExch(bar, 0u);          // ordered before the release below
        wide_red_release(bar + 1, 1u);
    }
    return g;
}
__device__ __forceinline__ bool wide_wait(unsigned *bar, unsigned g, int *flag, long long max_spin)
{
    long long it = 0;
    while (wide_ld_acquire(bar + 1) == g) {
        if (++it > max_spin) {
            atomicExch(flag + 1, 1);
            return false;
        }
    }
    return *(volatile int *)(flag + 1) == 0;
}

// value of a node array at index j in [-3, N+2] read from L2, with the parity ghosts
// u_{-k} = p0 u_k and u_{N-1+k} = p1 u_{N-1-k}
__device__ __forceinline__ double wide_ghost(const double *u, int N, int j, double p0, double p1)
{
    if (j < 0) return p0 * __ldcg(u - j);
    if (j > N - 1) return p1 * __ldcg(u + 2 * (N - 1) - j);
    return __ldcg(u + j);
}

// Phi-dot, Pi-dot at node j from the tiles (p, q, u point at node j's entries) and the stage
// update a_s y_n + b_s (y_s + dt L(y_s)) (a_0 = 0, b_0 = 1)
__device__ __forceinline__ void wide_update(const double *p, const double *q, const double *u, int j, int N,
                                            const InstDesc &d, double iT12, double as, double bs, double yn_P,
                                            double yn_Q, double &nP, double &nQ)
{
    const double kop = fma(-20.0, p[0], fma(15.0, add_f(p[-1], p[1]), fma(-6.0, add_f(p[-2], p[2]), add_f(p[-3], p[3]))));
    const double koq = fma(-20.0, q[0], fma(15.0, add_f(q[-1], q[1]), fma(-6.0, add_f(q[-2], q[2]), add_f(q[-3], q[3]))));
    double dP = 0.0, dQ = 0.0;
    if (j == 0) {
        dQ = fma(d.c3, fma(16.0, p[1], -2.0 * p[2]), mul_f(d.cko, koq));
    } else if (j < N - 1) {
        const double Df = fma(8.0, add_f(q[1], -q[-1]), add_f(q[-2], -q[2]));
        const double Du = fma(8.0, add_f(u[1], -u[-1]), add_f(u[-2], -u[2]));
        dP = fma(d.c12, Df, mul_f(d.cko, kop));
        dQ = fma(iT12, Du, mul_f(d.cko, koq));
    }
    const double sP = fma(d.dt, dP, p[0]), sQ = fma(d.dt, dQ, q[0]);
    nP = fma(as, yn_P, mul_f(bs, sP));
    nQ = fma(as, yn_Q, mul_f(bs, sQ));
}

__global__ void __launch_bounds__(kWideNT, 1) fixed_wide_kernel(WideArgs a)
{
    constexpr int NT = kWideNT, NB = kWideNodes, HW = kWideHalo, L = NB + 2 * HW;
    // tiles over the CTA's nodes and HW nodes on each side: entry k holds node i0 - HW + k;
    // Y[0]: y_n, Y[1]: y_1, Y[2]: y_2 (Phi, Pi); U: u = tan^2 x Phi of the stage slice being read
    __shared__ double Y[3][2][L];
    __shared__ double U[L];
    __shared__ double s_red[NT / 32];
    __shared__ int s_stop;
    const InstDesc &d = a.d;
    const int N = d.N, tid = threadIdx.x;
    const int i0 = blockIdx.x * NB, base = i0 - HW;
    const double aco[3] = {0.0, 0.75, 1.0 / 3.0}, bco[3] = {1.0, 0.25, 2.0 / 3.0};

    const long long step0 = a.st->step;
    const bool running = a.st->status == kRunning;
    const long long nsteps = (running && a.n_end > step0) ? a.n_end - step0 : 0;

    // own nodes of y_n (the other entries are copied after each barrier)
    for (int t = tid; t < NB; t += NT) {
        const int j = i0 + t;
        if (j < N) {
            Y[0][0][HW + t] = a.Phi[j];
            Y[0][1][HW + t] = a.Pi[j];
        }
    }
    __syncthreads();
    unsigned gen = 0;
    if (tid == 0) gen = wide_arrive(a.bar);
    bool pending = true;   // an arrival not yet waited for

    long long done = 0;
    for (long long n = 0; n < nsteps; ++n) {
        // every CTA's y_n is written (and the last slice was finite)
        if (tid == 0) {
            const bool w = wide_wait(a.bar, gen, a.flag, a.max_spin);
            s_stop = !w || __ldcg(a.flag) != 0;
        }
        __syncthreads();
        pending = false;
        if (s_stop) break;
        const double *gP = (n & 1) ? a.BP : a.Phi, *gQ = (n & 1) ? a.BQ : a.Pi;
        double *oP = (n & 1) ? a.Phi : a.BP, *oQ = (n & 1) ? a.Pi : a.BQ;
        // the entries no own node holds: nodes of the neighbouring CTAs and the parity ghosts
        // (Phi odd / even, Pi even / odd about 0 / pi/2) of nodes -3 .. -1 and N .. N+2
        for (int k = tid; k < L; k += NT) {
            const int j = base + k;
            const bool own = j >= i0 && j < i0 + NB && j < N;
            if (own || j < -3 || j > N + 2) continue;
            Y[0][0][k] = wide_ghost(gP, N, j, -1.0, 1.0);
            Y[0][1][k] = wide_ghost(gQ, N, j, 1.0, -1.0);
        }
        __syncthreads();
        for (int s = 0; s < 3; ++s) {
            const double (*ys)[L] = Y[s];
            double (*yo)[L] = Y[s < 2 ? s + 1 : 0];
            // u of y_s on the nodes the stage's stencils read: its range widened by 2; at pi/2 the
            // even extrapolation, beyond the ends the parity images (u odd / even about 0 / pi/2)
            const int ulo = base + 1 + 3 * s, uhi = i0 + NB + 8 - 3 * s;   // nodes [ulo, uhi)
            for (int t = tid; t < uhi - ulo; t += NT) {
                const int j = ulo + t;
                double v = 0.0;
                if (j >= -2 && j <= N + 1) {
                    auto u_at = [&](int x) { return mul_f(__ldg(a.T + x), ys[0][x - base]); };
                    if (j < 0) v = -u_at(-j);
                    else if (j < N - 1) v = u_at(j);
                    else if (j == N - 1) v = (4.0 * u_at(N - 2) - u_at(N - 3)) * (1.0 / 3.0);
                    else v = u_at(2 * (N - 1) - j);
                }
                U[j - base] = v;
            }
            __syncthreads();
            // the stage on nodes [i0 - 6 + 3s, i0 + NB + 6 - 3s) of the grid
            const int clo = i0 - 6 + 3 * s, chi = i0 + NB + 6 - 3 * s;
            const int j = clo + tid;
            const bool act = tid < chi - clo && j >= 0 && j < N;
            double nP = 0.0, nQ = 0.0;
            if (act) {
                const int k = j - base;
                wide_update(ys[0] + k, ys[1] + k, U + k, j, N, d, __ldg(a.iT12 + j), aco[s], bco[s], Y[0][0][k],
                            Y[0][1][k], nP, nQ);
            }
            __syncthreads();   // every read of Y[0] and U of this stage is done
            if (act) {
                const int k = j - base;
                yo[0][k] = nP;
                yo[1][k] = nQ;
                if (s == 2) {
                    oP[j] = nP;
                    oQ[j] = nQ;
                    if (!(isfinite(nP) && isfinite(nQ))) atomicExch(a.flag, 1);
                }
            }
            __syncthreads();
            if (s < 2) {
                // the parity ghosts of y_{s+1} next to both ends, from the nodes just formed
                for (int t = tid; t < 6; t += NT) {
                    const int jg = (t < 3) ? -1 - t : N + (t - 3);
                    const int jm = (t < 3) ? 1 + t : N - 2 - (t - 3);
                    const int kg = jg - base, km = jm - base;
                    if (kg >= 0 && kg < L && km >= 0 && km < L) {
                        yo[0][kg] = (t < 3) ? -yo[0][km] : yo[0][km];
                        yo[1][kg] = (t < 3) ? yo[1][km] : -yo[1][km];
                    }
                }
                __syncthreads();
            }
        }
        done = n + 1;
        if (tid == 0) gen = wide_arrive(a.bar);
        pending = true;
    }
    bool synced = true;
    if (pending) {   // the last arrival: every CTA has finished reading and writing the slices
        if (tid == 0) s_stop = !wide_wait(a.bar, gen, a.flag, a.max_spin);
        __syncthreads();
        synced = !s_stop;
    }
    // the final slice (step `done`) is in the second global slice after an odd number of steps:
    // its own nodes are copied back; the slice mass from the own nodes (the tile Y[0])
    double ms = 0.0;
    for (int t = tid; t < NB; t += NT) {
        const int j = i0 + t;
        if (j < N) {
            const double ph = Y[0][0][HW + t], pi = Y[0][1][HW + t];
            if (done & 1) {
                a.Phi[j] = ph;
                a.Pi[j] = pi;
            }
            ms = fma(__ldg(a.wsim + j), fma(ph, ph, mul_f(pi, pi)), ms);
        }
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
    __syncthreads();
    if (tid == 0) {
        gen = wide_arrive(a.bar);
        s_stop = !wide_wait(a.bar, gen, a.flag, a.max_spin);
    }
    __syncthreads();
    const bool synced2 = !s_stop;
    if (blockIdx.x == 0 && tid == 0) {
        double m = __ldcg(a.part);
        for (unsigned cb = 1; cb < gridDim.x; ++cb) m += __ldcg(a.part + cb);
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
