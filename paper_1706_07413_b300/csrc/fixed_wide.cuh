// fixed_wide.cuh -- one instance of the fixed-metric scheme evolved by the whole GPU.
//
// The paper's Table II case (Sec. IV): A = 1 and delta = 0 held fixed, so that Eqs. (eq:phi),
// (eq:pi) are the linear wave equation on AdS4, stepped with the Shu-Osher SSP-RK3 method.  The
// persistent kernels of evolve_ea.cuh give one instance at most one 16-CTA cluster (16 of the
// SMs); here a single instance is spread over a cooperative launch of ceil(N / kWideNT) CTAs, one
// grid node per thread, and the CTAs meet at one grid-wide barrier per Runge-Kutta stage:
//   stage s: each CTA holds its own nodes of the stage slice y_s and of u_s = tan^2 x Phi_s in
//            shared memory (it wrote them there in the previous stage); the nodes whose stencils
//            stay inside the block and away from the grid's ends form y_{s+1} = a_s y_n +
//            b_s (y_s + dt L(y_s)) at once, while the grid barrier that publishes y_s completes;
//            after it the block copies its 3-node halos (parity ghosts and u(pi/2) at the ends)
//            from L2, the remaining nodes are updated, and y_{s+1}, u_{s+1} are written to global
//            memory (for the neighbours' halos) and to the other shared tile, and the CTA arrives
//            at the next barrier.
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

// Phi-dot, Pi-dot at node i from the tile (p, q, u point at node i's entries) and the stage
// update y_{s+1} = a_s y_n + b_s (y_s + dt L(y_s)) (a_0 = 0, b_0 = 1)
__device__ __forceinline__ void wide_update(const double *p, const double *q, const double *u, int i, int N,
                                            const InstDesc &d, double iT12, double as, double bs, double yP,
                                            double yQ, double &nP, double &nQ)
{
    const double kop = fma(-20.0, p[0], fma(15.0, add_f(p[-1], p[1]), fma(-6.0, add_f(p[-2], p[2]), add_f(p[-3], p[3]))));
    const double koq = fma(-20.0, q[0], fma(15.0, add_f(q[-1], q[1]), fma(-6.0, add_f(q[-2], q[2]), add_f(q[-3], q[3]))));
    double dP = 0.0, dQ = 0.0;
    if (i == 0) {
        dQ = fma(d.c3, fma(16.0, p[1], -2.0 * p[2]), mul_f(d.cko, koq));
    } else if (i < N - 1) {
        const double Df = fma(8.0, add_f(q[1], -q[-1]), add_f(q[-2], -q[2]));
        const double Du = fma(8.0, add_f(u[1], -u[-1]), add_f(u[-2], -u[2]));
        dP = fma(d.c12, Df, mul_f(d.cko, kop));
        dQ = fma(iT12, Du, mul_f(d.cko, koq));
    }
    const double sP = fma(d.dt, dP, p[0]), sQ = fma(d.dt, dQ, q[0]);
    nP = fma(as, yP, mul_f(bs, sP));
    nQ = fma(as, yQ, mul_f(bs, sQ));
}

__global__ void __launch_bounds__(kWideNT, 1) fixed_wide_kernel(WideArgs a)
{
    constexpr int NT = kWideNT, H = 3, L = NT + 2 * H;
    // two tiles (the stage slice being read and the one being written) of Phi, Pi, u over the
    // block's nodes and a 3-node halo on each side: entry k holds node i0 - H + k
    __shared__ double tile[2][3][L];
    __shared__ double s_red[NT / 32];
    __shared__ int s_stop;
    const InstDesc &d = a.d;
    const int N = d.N, tid = threadIdx.x;
    const int i0 = blockIdx.x * NT, i = i0 + tid;
    const bool act = i < N;
    // nodes whose 7-point (Phi, Pi) and 5-point (u) stencils lie inside the block's own nodes and
    // need no parity ghost, the origin row or u(pi/2)
    const bool inner = act && tid >= H && tid < NT - H && i >= H && i <= N - 4;
    const double aco[3] = {0.0, 0.75, 1.0 / 3.0}, bco[3] = {1.0, 0.25, 2.0 / 3.0};
    const double Ti = act ? __ldg(a.T + i) : 0.0, iT12i = act ? __ldg(a.iT12 + i) : 0.0;

    const long long step0 = a.st->step;
    const bool running = a.st->status == kRunning;
    const long long nsteps = (running && a.n_end > step0) ? a.n_end - step0 : 0;

    // the slice y_n (own nodes, kept for the a_s y_n terms) and its u
    double yP = 0.0, yQ = 0.0;
    if (act) {
        yP = a.Phi[i];
        yQ = a.Pi[i];
        const double u = (i < N - 1) ? mul_f(Ti, yP) : 0.0;
        tile[0][0][tid + H] = yP;
        tile[0][1][tid + H] = yQ;
        tile[0][2][tid + H] = u;
        a.U0[i] = u;
    }
    __syncthreads();
    unsigned gen = 0;
    if (tid == 0) gen = wide_arrive(a.bar);
    bool pending = true;   // an arrival not yet waited for

    int c = 0, cu = 0;     // tile and global u buffer of the stage slice being read
    long long done = 0;
    bool ok = true;
    for (long long n = 0; n < nsteps && ok; ++n) {
        for (int s = 0; s < 3; ++s) {
            const double *gP = (s == 0) ? a.Phi : (s == 1) ? a.Y1P : a.Y2P;
            const double *gQ = (s == 0) ? a.Pi : (s == 1) ? a.Y1Q : a.Y2Q;
            const double *gU = cu ? a.U1 : a.U0;
            double *oP = (s == 0) ? a.Y1P : (s == 1) ? a.Y2P : a.Phi;
            double *oQ = (s == 0) ? a.Y1Q : (s == 1) ? a.Y2Q : a.Pi;
            double *oU = cu ? a.U0 : a.U1;
            double (*tc)[L] = tile[c];
            double nP = 0.0, nQ = 0.0;
            // the inner nodes, from the block's own values, while the barrier completes
            if (inner)
                wide_update(tc[0] + tid + H, tc[1] + tid + H, tc[2] + tid + H, i, N, d, iT12i, aco[s], bco[s], yP,
                            yQ, nP, nQ);
            // every CTA's y_s is written (and, at a step's first stage, the last slice was finite)
            if (tid == 0) {
                const bool w = wide_wait(a.bar, gen, a.flag, a.max_spin);
                s_stop = !w || (s == 0 && __ldcg(a.flag) != 0);
            }
            __syncthreads();
            pending = false;
            if (s_stop) { ok = false; break; }
            // the entries no own node holds: halos from the neighbouring blocks, parity ghosts
            // beyond both ends (Phi odd / even, Pi even / odd, u odd / even about 0 / pi/2) and
            // u(pi/2) by the even extrapolation
            for (int k = tid; k < L; k += NT) {
                const int j = i0 - H + k;
                if (j > N + 2) continue;
                const bool own = j >= i0 && j < i0 + NT && j < N;
                if (!own || j > N - 1) {
                    tc[0][k] = wide_ghost(gP, N, j, -1.0, 1.0);
                    tc[1][k] = wide_ghost(gQ, N, j, 1.0, -1.0);
                }
                if (!own || j >= N - 1)
                    tc[2][k] = (j == N - 1) ? (4.0 * __ldcg(gU + N - 2) - __ldcg(gU + N - 3)) * (1.0 / 3.0)
                                            : wide_ghost(gU, N, j, -1.0, 1.0);
            }
            __syncthreads();
            if (act && !inner)
                wide_update(tc[0] + tid + H, tc[1] + tid + H, tc[2] + tid + H, i, N, d, iT12i, aco[s], bco[s], yP,
                            yQ, nP, nQ);
            // y_{s+1} and u_{s+1} of the own nodes: global memory for the neighbours, the other tile
            if (act) {
                const double u = (i < N - 1) ? mul_f(Ti, nP) : 0.0;
                oP[i] = nP;
                oQ[i] = nQ;
                oU[i] = u;
                tile[c ^ 1][0][tid + H] = nP;
                tile[c ^ 1][1][tid + H] = nQ;
                tile[c ^ 1][2][tid + H] = u;
                if (s == 2) {
                    yP = nP;
                    yQ = nQ;
                    if (!(isfinite(nP) && isfinite(nQ))) atomicExch(a.flag, 1);
                }
            }
            __syncthreads();
            if (tid == 0) gen = wide_arrive(a.bar);
            pending = true;
            c ^= 1;
            cu ^= 1;
        }
        if (ok) done = n + 1;
    }
    bool synced = true;
    if (pending) {   // the last arrival: the final slice is complete everywhere
        if (tid == 0) s_stop = !wide_wait(a.bar, gen, a.flag, a.max_spin);
        __syncthreads();
        synced = !s_stop;
    }
    // the slice mass: per-CTA partial sums of the own nodes, then CTA 0 adds them in CTA order
    double ms = act ? mul_f(__ldg(a.wsim + i), fma(yP, yP, mul_f(yQ, yQ))) : 0.0;
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
