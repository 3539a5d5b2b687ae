// evolve.cuh -- persistent FP64 method-of-lines kernel for the AdS4 Einstein-Klein-Gordon
// system of arXiv:1706.07413, Sec. II (Eqs. (eq:phi), (eq:pi), (eq:aprime), (eq:delta)).
//
// One CTA -- or a thread-block cluster of CL = 2, 4, 8, 16 CTAs that split the node blocks between
// them -- evolves one instance at a time with its stage slice resident in (distributed) shared
// memory.  Thread t of a CTA owns the P contiguous grid nodes of its block and the cells to their
// right; node N-1 (x = pi/2, where Phi = Pi = 0) is owned by nobody and written as a constant.
// The kernel is instantiated for several (P, NT, CL) shapes; the host picks one per grid size.
//
// Per RK stage:
//   1. cell data: rho at nodes and (4-point interpolated) midpoints, the Simpson increment
//      Delta_c of Eq. (eq:delta) (in units of ln2/256, the reduction unit of the exponential)
//      and the RK4-in-x affine map m -> alpha_c m + beta_c of the mass-function form of
//      Eq. (eq:aprime);
//   2. a block scan: delta as a suffix sum of Delta, m as a prefix composition of affine maps
//      (per-thread serial, then warp shuffles, then one warp over the warp totals);
//   3. A = 1 - m cos^3 x / sin x, F = A e^{-delta}, fluxes f = F Pi and u = tan^2 x F Phi;
//   4. RHS: Phi-dot = D f, Pi-dot = D u / tan^2 x (Eq. (eq:pi) in its conservative form),
//      Kreiss-Oliger dissipation, classic RK4 accumulation into the other stage buffer.
// The FP64 pipe is the bound on this chip, so every term is arranged to minimise FP64
// instructions; comparisons, finiteness tests and indexing run on the integer pipe.
//
// Scheduling: work is cut into chunks of `chunk` RK4 steps of one instance.  Tickets are
// handed out in round-major order (round r, work item q); a chunk waits (bounded) for the
// previous chunk of the same instance to be released by whichever CTA ran it, so instances
// migrate between SMs and all SMs stay busy even when the batch is not a multiple of the SM
// count.  A CTA retires when fewer instances remain than CTAs take tickets, which keeps every
// wait shorter than about one chunk.  A wait that exceeds its iteration limit records an error
// and the CTAs leave; nothing spins without a bound.
//
// Shared-memory layout: node i of a field array lives at (i + 8) + (i + 8) / P, i.e. one pad
// double after every P nodes, so that the P-strided accesses of a warp hit distinct banks.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "expneg.cuh"

namespace adscl {

// per distinct grid size: geometry factors at nodes (length N) and cell midpoints (N-1); every
// table starts on a 16-byte boundary (tables are geo_stride(N) doubles apart), so that a thread's
// run of P factors is read with P/2 vector loads
struct GeoTab {
    const double *ws;    // h sin x cos x / 6
    const double *wt;    // h tan^2 x / 6            (0 at x = pi/2)
    const double *K;     // cos^3 x / sin x          (0 at both ends)
    const double *T;     // tan^2 x                  (0 at x = pi/2)
    const double *iT12;  // 1 / (12 h tan^2 x)       (0 at both ends)
    const double *wsm3;  // 3 h sin x cos x / (6*256) at x_{c+1/2}
    const double *wtm;   // h tan^2 x / (6*256)       at x_{c+1/2}
    const double *wsk;   // kappa ws, kappa = 256 / ln 2 (delta is accumulated in units of ln2/256)
    const double *iT12k; // iT12 / cq, cq = the dissipation factor of Pi-dot (sigma / (64 h), 1 if 0)
};

struct InstDesc {
    int32_t N;
    int32_t geo;
    int64_t off;  // offset of this instance in the packed field arrays
    double dt, dt2, dt3, dt6;
    double c12;   // 1 / (12 h)
    double c3;    // 3 / (12 h)
    double cko;   // sigma / (64 h)
    double rko;   // cko / c12 = 3 sigma / 16
    double dt6c, dt3c, dt2c, dtc;  // dt/6, dt/3, dt/2, dt times c12
    double dt6q, dt3q, dt2q, dtq;  // dt/6, dt/3, dt/2, dt times cq (Pi-dot is computed divided by cq)
    double c3q;   // c3 / cq
    int32_t ko;   // sigma > 0: dissipation on
    int32_t pad;
};

// distance in doubles between consecutive tables of one grid size: N rounded up to even
__host__ __device__ inline int geo_stride(int N) { return (N + 1) & ~1; }

// P consecutive doubles from a 16-byte aligned address, by P/2 vector loads on the read-only path
template <int P>
__device__ __forceinline__ void ldg_run(const double *p, double *v)
{
#pragma unroll
    for (int j = 0; j < P / 2; ++j) {
        const double2 x = __ldg(reinterpret_cast<const double2 *>(p) + j);
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
    }
}

// the per-instance coefficients above, for grid spacing h, step dt and dissipation sigma
__host__ inline void set_desc_coeffs(InstDesc &d, double h, double dt, double sigma)
{
    d.dt = dt;
    d.dt2 = 0.5 * dt;
    d.dt3 = dt / 3.0;
    d.dt6 = dt / 6.0;
    d.c12 = 1.0 / (12.0 * h);
    d.c3 = 3.0 / (12.0 * h);
    d.cko = sigma / (64.0 * h);
    d.rko = 3.0 * sigma / 16.0;
    d.dt6c = d.dt6 * d.c12;
    d.dt3c = d.dt3 * d.c12;
    d.dt2c = d.dt2 * d.c12;
    d.dtc = d.dt * d.c12;
    const double cq = sigma > 0.0 ? d.cko : 1.0;
    d.dt6q = d.dt6 * cq;
    d.dt3q = d.dt3 * cq;
    d.dt2q = d.dt2 * cq;
    d.dtq = d.dt * cq;
    d.c3q = d.c3 / cq;
    d.ko = sigma > 0.0 ? 1 : 0;
    d.pad = 0;
}
// iT12k of one node: 1 / (12 h T cq) = 16 / (3 sigma T) for sigma > 0 (0 where iT12 is 0)
__host__ __device__ inline double it12k_of(double h, double T, double sigma)
{
    return sigma > 0.0 ? 16.0 / (3.0 * sigma * T) : 1.0 / (12.0 * h * T);
}

enum : int32_t { kRunning = 0, kDone = 1, kCollapsed = 2, kNonfinite = 3, kTimeout = 4 };

struct InstState {
    int64_t step;   // index of the current slice (t = step * dt)
    double t_c;     // collapse time (+inf if none)
    double minA;    // min_x A of the current slice
    double mass;    // m(pi/2) of the current slice
    double delta0;  // delta(0) of the current slice
    int32_t status; // kRunning / kCollapsed / kNonfinite / kTimeout
    int32_t pad;
};

enum : int32_t { kModeEvolve = 0, kModeInit = 1, kModeSolve = 2 };

struct QueueCtl {
    int32_t ticket;      // next ticket
    int32_t unfinished;  // work items not yet finished in this launch
    int32_t active;      // CTAs still taking tickets
    int32_t error;       // 0, or 1 + work item whose wait ran out
};

constexpr int32_t kFinished = 0x7fffffff;

struct EvolveArgs {
    const InstDesc *desc;
    InstState *st;
    const GeoTab *geo;
    const double *exptab;  // 2^{j/256}, j < 256
    double *Phi, *Pi;      // packed current slices (updated in place)
    double *aPhi, *aPi;    // packed RK4 accumulators (workspace)
    const int32_t *order;  // work item -> instance
    int32_t nwork;
    int32_t chunk;         // RK4 steps per ticket
    int32_t max_rounds;    // tickets beyond nwork * max_rounds are never handed out
    int32_t mode;
    QueueCtl *ctl;
    int32_t *rounds;       // per work item: rounds completed, or kFinished
    long long max_spin;    // iteration limit of a wait
    double t_end;
    double theta;
    // kModeSolve only: packed A and delta of the slice (may be null); delta in units of ln2/256,
    // scaled by the caller, so that the node loop issues no multiplication for it
    double *outA, *outDelta;
    // kModeEvolve, optional (stage == null: off): the record of every stage of steps
    // 0 .. stage_steps-1 that the discrete adjoint sweeps backwards (see stage_slot)
    double *stage;
    long long stage_seg_stride;  // doubles between the buffers of consecutive segments
    long long stage_seg0;        // segment held by the first buffer
    long long stage_steps;
    int32_t stage_seg;           // steps per segment
    int32_t stage_nmax;          // node stride of one stored array
};

// Stage record: per stage s of step n of instance b, kStageArrays arrays of stage_nmax doubles:
// the stage input Phi, Pi (node N-1: 0), m and e^{-delta} and F = A e^{-delta} at the nodes
// (node N-1: M, 1, 1), alpha of the RK4-in-x map of m at the cells.  Segment g = n / stage_seg
// holds steps g stage_seg .. (g+1) stage_seg - 1 of every instance, in buffer g - stage_seg0.
constexpr int kStageArrays = 6;
__device__ __forceinline__ double *stage_slot(const EvolveArgs &a, int b, long long n, int s)
{
    const long long g = n / a.stage_seg, r = n - g * a.stage_seg;
    return a.stage + (g - a.stage_seg0) * a.stage_seg_stride +
           (((long long)b * a.stage_seg + r) * 4 + s) * kStageArrays * (long long)a.stage_nmax;
}

// order-preserving map of doubles onto signed 64-bit integers (integer-pipe min)
__device__ __forceinline__ long long order_key(double v) {
    long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double order_key_inv(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}
__device__ __forceinline__ bool is_finite_bits(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// offset of node (P*t + m) relative to the thread base (P+1)*t, for m >= -8
template <int P>
__device__ __forceinline__ constexpr int soff(int m) { return (m + 8) + (m + 8) / P; }
// absolute padded position of node i >= -8
template <int P>
__device__ __forceinline__ int spos(int i) { return (i + 8) + (i + 8) / P; }

// length of one padded shared-memory field array for grids up to Nmax nodes
template <int P>
__host__ __device__ constexpr int field_stride(int Nmax) {
    return (((Nmax + 12) + (Nmax + 12) / P + 1) + 1) & ~1;
}

static __global__ void queue_init_kernel(QueueCtl *ctl, int32_t *rounds, int nwork, int grid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ctl->ticket = 0;
        ctl->unfinished = nwork;
        ctl->active = grid;
        ctl->error = 0;
    }
    if (i < nwork) rounds[i] = 0;
}

// cluster-wide barrier for CL > 1 (every CTA of the cluster executes every barrier in the same
// order: all control decisions are taken by rank 0 and pushed to the others), CTA barrier for
// CL = 1
template <int CL>
__device__ __forceinline__ void csync() {
    if constexpr (CL > 1)
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else
        __syncthreads();
}
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
// stores into the same shared-memory location of CTA `dst` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void *p, int dst) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"((uint32_t)dst));
    return r;
}
__device__ __forceinline__ void st_peer(double *p, double v, int dst) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" :: "r"(peer_addr(p, dst)), "d"(v) : "memory");
}
__device__ __forceinline__ void st_peer(long long *p, long long v, int dst) {
    asm volatile("st.shared::cluster.b64 [%0], %1;" :: "r"(peer_addr(p, dst)), "l"(v) : "memory");
}
__device__ __forceinline__ void st_peer(int *p, int v, int dst) {
    asm volatile("st.shared::cluster.b32 [%0], %1;" :: "r"(peer_addr(p, dst)), "r"(v) : "memory");
}
// the same value into every other CTA of a CL-CTA cluster
template <int CL, class T>
__device__ __forceinline__ void st_others(T *p, T v, int rank) {
#pragma unroll
    for (int j = 1; j < CL; ++j) st_peer(p, v, (rank + j) % CL);
}
// first node block of cluster rank r when T node blocks are split over CL ranks
template <int CL>
__device__ __forceinline__ int block_start(int r, int T) { return (r * T + CL - 1) / CL; }

// CL = 1: one CTA per instance.  CL > 1: a cluster of CL CTAs per instance (built for 2, 4, 8, 9
// and 16; 9 and 16 are non-portable cluster sizes, allowed per kernel by the host), rank r owning
// the node blocks block_start(r) .. block_start(r+1)-1 (at least NT/2 blocks each, so P >= 3
// halo nodes always come from the neighbouring rank); halos, scan carries and the step-end
// diagnostics cross between the CTAs through distributed shared memory.
// launch bounds: 512 threads per SM worth of CTAs (one CTA of 512, two of 256, four of 128), so
// that every shape gets the same 128 registers per thread
// REC: the variant that also writes the stage record (EvolveArgs::stage) for the adjoint
template <int P, int NT, int CL = 1, bool REC = false>
__global__ void __launch_bounds__(NT, (NT >= 512) ? 1 : 512 / NT) evolve_kernel(EvolveArgs a, int stride)
{
    static_assert(P >= 4 && (P & (P - 1)) == 0, "P: power of two >= 4");
    static_assert(CL >= 1 && CL <= 16, "cluster of 1 to 16 CTAs");
    constexpr int NW = NT / 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ double smem[];
    double *bufA0 = smem, *bufA1 = smem + stride;                   // stage Phi, Pi
    double *bufB0 = smem + 2 * stride, *bufB1 = smem + 3 * stride;  // next stage Phi, Pi
    double *sF = smem + 4 * stride, *sU = smem + 5 * stride;        // alpha/beta, then f/u
    __shared__ double s_tab[kExpTableSize];
    __shared__ double wAl[NW], wBe[NW], wDe[NW], cM[NW], cMa[NW], cD[NW];
    __shared__ long long wMin[NW], wMinP[CL * NW];
    __shared__ double s_mass, s_d0, s_cA[CL], s_cB[CL], s_cD[CL];
    __shared__ int s_cmd, s_q, s_r, s_leave;
    __shared__ long long s_step;
    __shared__ double s_tc, s_minA, s_massS, s_d0S;
    __shared__ int s_status;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int rank = 0;
    if constexpr (CL > 1) rank = cluster_rank();
    for (int i = tid; i < kExpTableSize; i += NT) s_tab[i] = a.exptab[i];
    csync<CL>();   // every CTA of the cluster has started before any remote shared-memory store

    for (;;) {
        // ------------------------------------------------------------ take a ticket
        if (tid == 0 && rank == 0) {
            int cmd = 0, q = 0, r = 0;  // cmd 0: leave, 1: run
            for (;;) {
                if (ld_relaxed(&a.ctl->unfinished) == 0 || ld_relaxed(&a.ctl->error) != 0) break;
                const int t = atomicAdd(&a.ctl->ticket, 1);
                if (t >= a.nwork * a.max_rounds) break;
                r = t / a.nwork;
                q = t - r * a.nwork;
                int rd = ld_acquire(a.rounds + q);
                long long spin = 0;
                while (rd < r) {  // the previous chunk of this instance is still running
                    if (++spin > a.max_spin) break;
                    __nanosleep(256);
                    rd = ld_acquire(a.rounds + q);
                }
                if (rd == kFinished) continue;
                if (rd < r) {
                    atomicCAS(&a.ctl->error, 0, q + 1);
                    break;
                }
                cmd = 1;
                break;
            }
            InstState S{};
            if (cmd) {
                const InstState *sp = a.st + a.order[q];
                S.step = __ldcg(&sp->step);
                S.t_c = __ldcg(&sp->t_c);
                S.minA = __ldcg(&sp->minA);
                S.mass = __ldcg(&sp->mass);
                S.delta0 = __ldcg(&sp->delta0);
                S.status = __ldcg(&sp->status);
            }
            s_cmd = cmd;
            s_q = q;
            s_r = r;
            s_step = S.step;
            s_tc = S.t_c;
            s_minA = S.minA;
            s_massS = S.mass;
            s_d0S = S.delta0;
            s_status = S.status;
            if constexpr (CL > 1) {
                st_others<CL>(&s_cmd, cmd, 0);
                st_others<CL>(&s_q, q, 0);
                st_others<CL>(&s_r, r, 0);
                st_others<CL>(&s_step, (long long)S.step, 0);
                st_others<CL>(&s_tc, S.t_c, 0);
                st_others<CL>(&s_minA, S.minA, 0);
                st_others<CL>(&s_massS, S.mass, 0);
                st_others<CL>(&s_d0S, S.delta0, 0);
                st_others<CL>(&s_status, (int)S.status, 0);
            }
        }
        csync<CL>();
        if (s_cmd == 0) break;
        const int q = s_q, rnd = s_r;
        const int b = a.order[q];
        const InstDesc d = a.desc[b];
        InstState S;
        S.step = s_step;
        S.t_c = s_tc;
        S.minA = s_minA;
        S.mass = s_massS;
        S.delta0 = s_d0S;
        S.status = s_status;

        const double dt = d.dt;
        long long n_end = S.step, n_target = S.step;
        if (a.mode == kModeEvolve) {
            n_end = (long long)ceil(a.t_end / dt - 1e-9);
            n_target = min(n_end, S.step + (long long)a.chunk);
        }
        const int N = d.N;
        const int TnAll = (N - 1) / P;
        const int bs = block_start<CL>(rank, TnAll);
        const int Tn = block_start<CL>(rank + 1, TnAll) - bs;  // node blocks of this CTA
        const int gb = bs * P;                                  // first node of this CTA
        const int NLp = (rank > 0) ? (bs - block_start<CL>(rank - 1, TnAll)) * P : 0;  // nodes of rank-1
        const bool act = tid < Tn;
        const bool tfirst = rank == 0 && tid == 0;              // owns node 0
        const bool last = (rank == CL - 1) && tid == Tn - 1;    // owns node N-2
        const bool hl = (CL > 1) && rank < CL - 1 && tid == Tn - 1;  // pushes the left halo of rank+1
        const bool hr = (CL > 1) && rank > 0 && tid == 0;            // pushes the right halo of rank-1
        const int i0 = gb + tid * P;       // global node of the thread's first node
        const int tb = (P + 1) * tid;      // thread base in the padded arrays (local nodes)
        const int Nl = N - gb;             // local index of node N (boundary ghosts: Nl - 1 + j)
        const GeoTab g = a.geo[d.geo];
        double *uPhi = a.Phi + d.off, *uPi = a.Pi + d.off;
        double *cPhi = a.aPhi + d.off, *cPi = a.aPi + d.off;
        const bool skip = (a.mode == kModeEvolve) && (S.status != kRunning || S.step >= n_target);

        long long step = S.step;
        double minA_prev = S.minA, minA = S.minA, mass = S.mass, d0 = S.delta0, t_c = S.t_c;
        int32_t status = S.status;

        if (!skip) {
            // ---- load the current slice into stage buffer A (boundary values imposed) ----
            if (act) {
                double p[P], qv[P];
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    p[k] = __ldcg(uPhi + i0 + k);
                    qv[k] = __ldcg(uPi + i0 + k);
                }
                if (tfirst) p[0] = 0.0;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    bufA0[tb + soff<P>(k)] = p[k];
                    bufA1[tb + soff<P>(k)] = qv[k];
                }
                if (tfirst) {
#pragma unroll
                    for (int j = 1; j <= 3; ++j) {
                        bufA0[spos<P>(-j)] = -p[j];
                        bufA1[spos<P>(-j)] = qv[j];
                    }
                    if (a.mode == kModeInit) uPhi[0] = 0.0;
                }
                if (last) {
                    bufA0[spos<P>(Nl - 1)] = 0.0;
                    bufA1[spos<P>(Nl - 1)] = 0.0;
#pragma unroll
                    for (int j = 1; j <= 3; ++j) {
                        bufA0[spos<P>(Nl - 1 + j)] = p[P - j];
                        bufA1[spos<P>(Nl - 1 + j)] = -qv[P - j];
                    }
                    if (a.mode == kModeInit) {
                        uPhi[N - 1] = 0.0;
                        uPi[N - 1] = 0.0;
                    }
                }
                if constexpr (CL > 1) {
                    if (hl) {   // last 3 nodes -> left halo of rank+1
#pragma unroll
                        for (int j = 1; j <= 3; ++j) {
                            st_peer(bufA0 + spos<P>(-j), p[P - j], rank + 1);
                            st_peer(bufA1 + spos<P>(-j), qv[P - j], rank + 1);
                        }
                    }
                    if (hr) {   // first 3 nodes -> right halo of rank-1
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            st_peer(bufA0 + spos<P>(NLp + j), p[j], rank - 1);
                            st_peer(bufA1 + spos<P>(NLp + j), qv[j], rank - 1);
                        }
                    }
                }
            }
            csync<CL>();

            double *S0 = bufA0, *S1 = bufA1, *D0 = bufB0, *D1 = bufB1;
            bool first = true;
            for (;;) {
#pragma unroll 1
                for (int s = 0; s < 4; ++s) {
                    // stage record for the adjoint (REC): its address is recomputed where it is
                    // written (short live range)
                    const bool rec = REC && step < a.stage_steps;
                    // ================= constraint solve on the stage slice =================
                    double De[P];
                    double aT = 1.0, bT = 0.0, SD = 0.0;
                    if (act) {
                        double *stg = nullptr;
                        if constexpr (REC) stg = rec ? stage_slot(a, b, step, s) : nullptr;
                        const int snm = a.stage_nmax;
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        double pm1 = Sp[soff<P>(-1)], p0 = Sp[soff<P>(0)], p1 = Sp[soff<P>(1)];
                        double qm1 = Sq[soff<P>(-1)], q0 = Sq[soff<P>(0)], q1 = Sq[soff<P>(1)];
                        // geometry of the thread's nodes i0 .. i0+P and cells i0 .. i0+P-1
                        double gws[P + 1], gwt[P + 1], gwm[P], gtm[P];
                        ldg_run<P>(g.wsk + i0, gws);
                        ldg_run<P>(g.wt + i0, gwt);
                        ldg_run<P>(g.wsm3 + i0, gwm);
                        ldg_run<P>(g.wtm + i0, gtm);
                        gws[P] = __ldg(g.wsk + i0 + P);
                        gwt[P] = __ldg(g.wt + i0 + P);
                        const double rho0 = fma(p0, p0, mul_f(q0, q0));
                        double qn0 = mul_f(gws[0], rho0), rn0 = mul_f(gwt[0], rho0);
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const double p2 = Sp[soff<P>(k + 2)], q2 = Sq[soff<P>(k + 2)];
                            const double rho1 = fma(p1, p1, mul_f(q1, q1));
                            const double qn1 = mul_f(gws[k + 1], rho1);   // kappa q1
                            const double rn1 = mul_f(gwt[k + 1], rho1);
                            // 16 * (midpoint value) by the 4-point Lagrange formula
                            const double p16 = fma(9.0, add_f(p0, p1), -add_f(pm1, p2));
                            const double q16 = fma(9.0, add_f(q0, q1), -add_f(qm1, q2));
                            const double rm = fma(p16, p16, mul_f(q16, q16));  // 256 rho_{c+1/2}
                            const double qm3 = mul_f(gwm[k], rm);   // 3 (h s rho / 6) at the midpoint
                            const double tm = mul_f(gtm[k], rm);    // h tan^2 rho / 6 there
                            const double s01 = add_f(qn0, qn1);               // kappa (q0 + q1)
                            // Simpson increment of delta over the cell, in units of ln2/256
                            const double dek = fma(kKappa * (4.0 / 3.0), qm3, s01);
                            // RK4 in x of m' = a - b m over the cell as the affine map
                            // m -> alpha m + beta (alpha: y' = -b y, y(0) = 1; beta: y' = a - b y,
                            // y(0) = 0).  With q = h b / 6 and r = h a / 6 at the cell's left end
                            // (q0, r0), midpoint (qm, tm) and right end (q1, r1), the stages give
                            //   alpha = 1 - q0 - q1 - 2 qm (Y2 + Y3) + 6 qm q1 Y3,
                            //   Y2 = 1 - 3 q0, Y3 = 1 - 3 qm Y2;
                            //   beta = r0 + r1 + 2 W2 + W3 (2 - 6 q1),
                            //   W2 = tm - 3 qm r0, W3 = tm - 3 qm W2.
                            // Eliminating Y2 and W3 (3 qm Y2 = 1 - Y3):
                            //   alpha = (1/3 - q0 - q1) + y3 e,   beta = (r0 + r1) + ca tm + e W2,
                            //   y3 = Y3 / 3 = 1/3 - 3 qm (1/3 - q0), ca = 2 - 6 q1, e = 2 - 3 qm ca.
                            const double y2 = fma(-kInvKappa, qn0, 1.0 / 3.0);       // 1/3 - q0
                            const double y3 = fma(-qm3, y2, 1.0 / 3.0);
                            const double ca = fma(-6.0 * kInvKappa, qn1, 2.0);       // 2 - 6 q1
                            const double e = fma(-qm3, ca, 2.0);
                            const double al = fma(y3, e, fma(-kInvKappa, s01, 1.0 / 3.0));
                            const double w2 = fma(-qm3, rn0, tm);
                            const double be = fma(e, w2, fma(ca, tm, add_f(rn0, rn1)));
                            if (stg) {
                                stg[i0 + k] = p0;
                                stg[snm + i0 + k] = q0;
                                stg[5 * snm + i0 + k] = al;
                            }
                            // running compositions: (aT, bT) maps m at node i0 to m at node i0+k+1,
                            // De[k] = sum of the increments of cells i0 .. i0+k-1 (k >= 1); both
                            // let the flux phase form every node's m and delta independently
                            if (k == 0) {
                                aT = al;
                                bT = be;
                                SD = dek;
                            } else {
                                bT = fma(al, bT, be);
                                aT = mul_f(aT, al);
                                De[k] = SD;
                                SD = add_f(SD, dek);
                            }
                            if (k < P - 1) {
                                sF[tb + soff<P>(k + 1)] = aT;
                                sU[tb + soff<P>(k + 1)] = bT;
                            }
                            pm1 = p0; p0 = p1; p1 = p2;
                            qm1 = q0; q0 = q1; q1 = q2;
                            qn0 = qn1; rn0 = rn1;
                        }
                        if (stg && last) {
                            stg[N - 1] = 0.0;
                            stg[snm + N - 1] = 0.0;
                        }
                    }
                    // warp-level inclusive scans: affine prefix (lanes ascending), delta suffix sum
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const double ap = __shfl_up_sync(FULL, aT, o);
                        const double bp = __shfl_up_sync(FULL, bT, o);
                        const double dn = __shfl_down_sync(FULL, SD, o);
                        if (lane >= o) {
                            bT = fma(aT, bp, bT);
                            aT = mul_f(aT, ap);
                        }
                        if (lane + o < 32) SD = add_f(SD, dn);
                    }
                    double aEx = __shfl_up_sync(FULL, aT, 1);
                    double bEx = __shfl_up_sync(FULL, bT, 1);
                    if (lane == 0) { aEx = 1.0; bEx = 0.0; }
                    if (lane == 31) { wAl[wid] = aT; wBe[wid] = bT; }
                    if (lane == 0) wDe[wid] = SD;
                    __syncthreads();
                    if (wid == 0) {
                        double A_ = lane < NW ? wAl[lane] : 1.0;
                        double B_ = lane < NW ? wBe[lane] : 0.0;
                        double D_ = lane < NW ? wDe[lane] : 0.0;
#pragma unroll
                        for (int o = 1; o < NW; o <<= 1) {
                            const double ap = __shfl_up_sync(FULL, A_, o);
                            const double bp = __shfl_up_sync(FULL, B_, o);
                            const double dn = __shfl_down_sync(FULL, D_, o);
                            if (lane >= o) {
                                B_ = fma(A_, bp, B_);
                                A_ = A_ * ap;
                            }
                            if (lane + o < NW) D_ = D_ + dn;
                        }
                        double bw = __shfl_up_sync(FULL, B_, 1);
                        double dw = __shfl_down_sync(FULL, D_, 1);
                        if (lane == 0) bw = 0.0;
                        if (lane + 1 >= NW) dw = 0.0;
                        if (lane < NW) { cM[lane] = bw; cD[lane] = dw; }
                        if constexpr (CL > 1) {
                            double aw = __shfl_up_sync(FULL, A_, 1);
                            if (lane == 0) aw = 1.0;
                            if (lane < NW) cMa[lane] = aw;
                            // block totals to the other ranks: the m map to higher ranks, the delta
                            // sum to lower ranks (slot = the sender's rank)
                            if (lane == NW - 1) {
                                for (int j = rank + 1; j < CL; ++j) {
                                    st_peer(s_cA + rank, A_, j);
                                    st_peer(s_cB + rank, B_, j);
                                }
                            }
                            if (lane == 0) {
                                for (int j = 0; j < rank; ++j) st_peer(s_cD + rank, D_, j);
                            }
                        }
                    }
                    csync<CL>();

                    long long kmin = 0x7FFFFFFFFFFFFFFFLL;
                    if (act) {
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        double *stg = nullptr;
                        if constexpr (REC) stg = rec ? stage_slot(a, b, step, s) : nullptr;
                        const int snm = a.stage_nmax;
                        // m at the warp's first node (cm) and at node i0 (m); delta at node i0 (dtop) from
                        // the inclusive suffix sum SD of this and the warp's later lanes
                        double m, cm, dtop;
                        if constexpr (CL > 1) {
                            // m at this rank's first node: the maps of ranks 0 .. rank-1 applied to m = 0
                            double mr = 0.0;
                            for (int j = 0; j < rank; ++j) mr = (j == 0) ? s_cB[0] : fma(s_cA[j], mr, s_cB[j]);
                            // delta carried in from the ranks to the right
                            double dr = 0.0;
                            for (int j = CL - 1; j > rank; --j) dr = (j == CL - 1) ? s_cD[j] : dr + s_cD[j];
                            cm = (rank > 0) ? fma(cMa[wid], mr, cM[wid]) : cM[wid];
                            m = fma(aEx, cm, bEx);
                            dtop = SD + cD[wid] + ((rank < CL - 1) ? dr : 0.0);
                        } else {
                            cm = cM[wid];
                            m = fma(aEx, cm, bEx);
                            dtop = SD + cD[wid];
                        }
                        // delta at node i0+k: dtop minus the increments of the cells i0 .. i0+k-1
                        De[0] = dtop;
#pragma unroll
                        for (int k = 1; k < P; ++k) De[k] = add_f(dtop, -De[k]);
                        double g1 = 0.0, g2 = 0.0, um1 = 0.0, um2 = 0.0, fm1 = 0.0, fm2 = 0.0;
                        double f0 = 0.0, f1 = 0.0, u0 = 0.0, u1 = 0.0;
                        double gK[P], gT[P];
                        ldg_run<P>(g.K + i0, gK);
                        ldg_run<P>(g.T + i0, gT);
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int i = i0 + k;
                            const double mk = (k == 0) ? m : fma(sF[tb + soff<P>(k)], m, sU[tb + soff<P>(k)]);
                            const double Ai = fma(-mk, gK[k], 1.0);
                            kmin = min_ll(kmin, order_key(Ai));
                            const double Ei = a_exp_neg_scaled(1.0, De[k], s_tab);   // e^{-delta}
                            const double Fi = mul_f(Ai, Ei);
                            if (stg) {
                                stg[2 * snm + i] = mk;
                                stg[3 * snm + i] = Ei;
                                stg[4 * snm + i] = Fi;
                            }
                            const double gi = mul_f(Fi, Sp[soff<P>(k)]);
                            const double fi = mul_f(Fi, Sq[soff<P>(k)]);
                            const double ui = mul_f(gT[k], gi);
                            sF[tb + soff<P>(k)] = fi;
                            sU[tb + soff<P>(k)] = ui;
                            if (k == 0) { f0 = fi; u0 = ui; }
                            if (k == 1) { g1 = gi; f1 = fi; u1 = ui; }
                            if (k == 2) g2 = gi;
                            if (tfirst && (k == 1 || k == 2)) {
                                sF[spos<P>(-k)] = fi;   // f = F Pi: even about x = 0
                                sU[spos<P>(-k)] = neg_bits(ui);  // u = tan^2 F Phi: odd about x = 0
                            }
                            if (k == P - 1) { fm1 = fi; um1 = ui; }
                            if (k == P - 2) { fm2 = fi; um2 = ui; }
                            if (a.outA) {
                                a.outA[d.off + i] = Ai;
                                a.outDelta[d.off + i] = De[k];   // in units of ln2/256 (no FP64 work here)
                            }
                        }
                        // the grid's two ends, in a branch that only their warps take (a vote result is
                        // uniform over the warp), so the other warps issue none of this FP64 work
                        if (__any_sync(__activemask(), tfirst || last)) {
                        if (last) {
                            const double mN = fma(aT, cm, bT);   // m at node N-1: the inclusive prefix map
                            s_mass = mN;
                            if (stg) {
                                stg[2 * snm + N - 1] = mN;
                                stg[3 * snm + N - 1] = 1.0;
                                stg[4 * snm + N - 1] = 1.0;
                            }
                        }
                        if (tfirst) {
                            const double d0n = De[0] * kInvKappa;   // delta(0)
                            s_d0 = d0n;
                            // Pi-dot at x = 0 needs (F Phi)'(0) = (16 g_1 - 2 g_2) / (12 h)
                            sF[spos<P>(-3)] = fma(16.0, g1, -2.0 * g2);
                            if constexpr (CL > 1) st_others<CL>(&s_d0, d0n, 0);
                        }
                        if (last) {
                            // f odd and u even about x = pi/2; u(pi/2) by even extrapolation
                            sF[spos<P>(Nl - 1)] = 0.0;
                            sF[spos<P>(Nl)] = neg_bits(fm1);
                            sF[spos<P>(Nl + 1)] = neg_bits(fm2);
                            sU[spos<P>(Nl - 1)] = (4.0 * um1 - um2) * (1.0 / 3.0);
                            sU[spos<P>(Nl)] = um1;
                            sU[spos<P>(Nl + 1)] = um2;
                            if (a.outA) {
                                a.outA[d.off + N - 1] = 1.0;
                                a.outDelta[d.off + N - 1] = 0.0;
                            }
                            if constexpr (CL > 1) st_others<CL>(&s_mass, s_mass, CL - 1);
                        }
                        }
                        if constexpr (CL > 1) {
                            if (hl) {   // f, u at the last 2 nodes -> left halo of rank+1
                                st_peer(sF + spos<P>(-1), fm1, rank + 1);
                                st_peer(sF + spos<P>(-2), fm2, rank + 1);
                                st_peer(sU + spos<P>(-1), um1, rank + 1);
                                st_peer(sU + spos<P>(-2), um2, rank + 1);
                            }
                            if (hr) {   // f, u at the first 2 nodes -> right halo of rank-1
                                st_peer(sF + spos<P>(NLp), f0, rank - 1);
                                st_peer(sF + spos<P>(NLp + 1), f1, rank - 1);
                                st_peer(sU + spos<P>(NLp), u0, rank - 1);
                                st_peer(sU + spos<P>(NLp + 1), u1, rank - 1);
                            }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) kmin = min_ll(kmin, __shfl_xor_sync(FULL, kmin, o));
                    if (lane == 0) {
                        wMin[wid] = kmin;
                        if constexpr (CL > 1) st_others<CL>(wMinP + rank * NW + wid, kmin, rank);
                    }
                    csync<CL>();

                    if (s == 0) {
                        // ---------- end-of-step diagnostics on the slice t = step * dt ----------
                        long long km = wMin[0];
#pragma unroll
                        for (int w = 1; w < NW; ++w) km = min_ll(km, wMin[w]);
                        if constexpr (CL > 1) {
                            for (int j = 1; j < CL; ++j) {
                                const long long *wp = wMinP + ((rank + j) % CL) * NW;
#pragma unroll
                                for (int w = 0; w < NW; ++w) km = min_ll(km, wp[w]);
                            }
                        }
                        minA = order_key_inv(km);
                        mass = s_mass;
                        d0 = s_d0;
                        const bool nonfin = !(is_finite_bits(mass) && is_finite_bits(d0));
                        bool stop = false;
                        if (a.mode != kModeEvolve) {
                            if (a.mode == kModeInit) {
                                status = nonfin ? kNonfinite : (minA < a.theta ? kCollapsed : kRunning);
                                t_c = (status == kCollapsed) ? 0.0
                                                             : __longlong_as_double(0x7FF0000000000000LL);
                            }
                            stop = true;
                        } else if (!first) {
                            if (nonfin) {
                                status = kNonfinite;
                                stop = true;
                            } else if (minA < a.theta) {
                                // min A crossed theta between t_{n-1} and t_n: linear interpolation
                                t_c = (double)(step - 1) * dt +
                                      dt * (minA_prev - a.theta) / (minA_prev - minA);
                                status = kCollapsed;
                                stop = true;
                            }
                        }
                        if (!stop && step >= n_target) stop = true;
                        if (stop) goto finish;
                        minA_prev = minA;
                        first = false;
                    }

                    // ================= right-hand side and RK4 update =================
                    if (act) {
                        const double wacc = (s == 0 || s == 3) ? d.dt6q : d.dt3q;
                        const double wst = (s == 2) ? d.dtq : d.dt2q;
                        const double waccc = (s == 0 || s == 3) ? d.dt6c : d.dt3c;
                        const double wstc = (s == 2) ? d.dtc : d.dt2c;
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        const double *f = sF + tb, *u = sU + tb;
                        double *Dp = D0 + tb, *Dq = D1 + tb;
                        double gI[P];
                        ldg_run<P>(g.iT12k + i0, gI);
                        // the node loop, compiled once per stage kind (first, middle, last) so that no stage
                        // issues another's FP64 work with its lanes predicated off
                        auto update_nodes = [&](auto stage_kind) {
                        constexpr int KIND = decltype(stage_kind)::value;
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int i = i0 + k;
                            const double Df = fma(8.0, add_f(f[soff<P>(k + 1)], -f[soff<P>(k - 1)]),
                                                  add_f(f[soff<P>(k - 2)], -f[soff<P>(k + 2)]));
                            const double Du = fma(8.0, add_f(u[soff<P>(k + 1)], -u[soff<P>(k - 1)]),
                                                  add_f(u[soff<P>(k - 2)], -u[soff<P>(k + 2)]));
                            const double kp = fma(-20.0, Sp[soff<P>(k)],
                                fma(15.0, add_f(Sp[soff<P>(k - 1)], Sp[soff<P>(k + 1)]),
                                fma(-6.0, add_f(Sp[soff<P>(k - 2)], Sp[soff<P>(k + 2)]),
                                    add_f(Sp[soff<P>(k - 3)], Sp[soff<P>(k + 3)]))));
                            const double kq = fma(-20.0, Sq[soff<P>(k)],
                                fma(15.0, add_f(Sq[soff<P>(k - 1)], Sq[soff<P>(k + 1)]),
                                fma(-6.0, add_f(Sq[soff<P>(k - 2)], Sq[soff<P>(k + 2)]),
                                    add_f(Sq[soff<P>(k - 3)], Sq[soff<P>(k + 3)]))));
                            // Phi-dot = c12 (Df + rko kp) and Pi-dot = cq (iT12k Du + kq): the factors
                            // c12 and cq are folded into the RK weights
                            // at node 0: Phi(0) = 0 and Pi-dot = 3 (F Phi)'(0) / cq, chosen by operand
                            // and result selects so that no thread issues a predicated-off FMA
                            const bool origin = (k == 0) && tfirst;
                            const double kqs = d.ko ? kq : 0.0;
                            const double Xp = origin ? 0.0 : fma(d.rko, kp, Df);
                            const double dQ = fma(origin ? d.c3q : gI[k], origin ? sF[spos<P>(-3)] : Du, kqs);
                            // the slice u_n: the stage itself at s = 0, from global memory at
                            // s = 1, 2, not needed at s = 3
                            double up = 0.0, uq = 0.0;
                            if constexpr (KIND == 0) {
                                up = Sp[soff<P>(k)];
                                uq = Sq[soff<P>(k)];
                            } else if constexpr (KIND == 1) {
                                up = __ldcg(uPhi + i);
                                uq = __ldcg(uPi + i);
                            }
                            // RK4 accumulators in a node-block-interleaved layout (entry k of node
                            // block t at k * TnAll + t), so that a warp's accesses are contiguous
                            const int ci = k * TnAll + bs + tid;
                            double ap_, aq_;
                            if constexpr (KIND == 0) {
                                ap_ = fma(waccc, Xp, up);
                                aq_ = fma(wacc, dQ, uq);
                            } else {
                                ap_ = fma(waccc, Xp, __ldcg(cPhi + ci));
                                aq_ = fma(wacc, dQ, __ldcg(cPi + ci));
                            }
                            double np, nq;
                            if constexpr (KIND < 2) {
                                cPhi[ci] = ap_;
                                cPi[ci] = aq_;
                                np = fma(wstc, Xp, up);
                                nq = fma(wst, dQ, uq);
                            } else {
                                np = ap_;
                                nq = aq_;
                                uPhi[i] = ap_;
                                uPi[i] = aq_;
                            }
                            Dp[soff<P>(k)] = np;
                            Dq[soff<P>(k)] = nq;
                            if (tfirst && k >= 1 && k <= 3) {
                                D0[spos<P>(-k)] = neg_bits(np);  // Phi odd about x = 0
                                D1[spos<P>(-k)] = nq;   // Pi even about x = 0
                            }
                            if (last && k >= P - 3) {
                                D0[spos<P>(Nl - 1 + (P - k))] = np;   // Phi even about pi/2
                                D1[spos<P>(Nl - 1 + (P - k))] = neg_bits(nq);  // Pi odd about pi/2
                            }
                            if constexpr (CL > 1) {
                                if (hl && k >= P - 3) {      // -> left halo of rank+1
                                    st_peer(D0 + spos<P>(-(P - k)), np, rank + 1);
                                    st_peer(D1 + spos<P>(-(P - k)), nq, rank + 1);
                                }
                                if (hr && k < 3) {           // -> right halo of rank-1
                                    st_peer(D0 + spos<P>(NLp + k), np, rank - 1);
                                    st_peer(D1 + spos<P>(NLp + k), nq, rank - 1);
                                }
                            }
                        }
                        };
                        if (s == 0) update_nodes(std::integral_constant<int, 0>{});
                        else if (s < 3) update_nodes(std::integral_constant<int, 1>{});
                        else update_nodes(std::integral_constant<int, 2>{});
                        if (last) {
                            D0[spos<P>(Nl - 1)] = 0.0;
                            D1[spos<P>(Nl - 1)] = 0.0;
                        }
                    }
                    csync<CL>();
                    double *t0 = S0, *t1 = S1;
                    S0 = D0; S1 = D1; D0 = t0; D1 = t1;
                }
                ++step;
            }
        }
    finish:
        csync<CL>();  // all global writes of this chunk are issued, by every CTA of the cluster
        if (tid == 0 && rank == 0) {
            if (!skip) {
                InstState *sp = a.st + b;
                sp->step = step;
                sp->t_c = t_c;
                sp->minA = minA;
                sp->mass = mass;
                sp->delta0 = d0;
                sp->status = status;
            }
            __threadfence();
            const bool fin = (a.mode != kModeEvolve) || status != kRunning || step >= n_end;
            if (fin) {
                atomicExch(a.rounds + q, kFinished);
                atomicSub(&a.ctl->unfinished, 1);
            } else {
                atomicExch(a.rounds + q, rnd + 1);
            }
            // retire when fewer work items remain than CTAs (clusters) take tickets
            int leave = 0;
            for (;;) {
                const int act_n = ld_relaxed(&a.ctl->active);
                const int unf = ld_relaxed(&a.ctl->unfinished);
                if (unf >= act_n) break;
                if (atomicCAS(&a.ctl->active, act_n, act_n - 1) == act_n) {
                    leave = 1;
                    break;
                }
            }
            s_leave = leave;
            if constexpr (CL > 1) st_others<CL>(&s_leave, leave, 0);
        }
        csync<CL>();
        if (s_leave) break;
    }
}

// per-instance results of an evolve call: t_reached, t_collapse, mass, status
// (with ctl given, the instance whose chunk wait ran out in that launch is reported as kTimeout)
static __global__ void gather_kernel(const InstDesc *desc, const InstState *st, int B, double t_end,
                              int evolve_call, const QueueCtl *ctl, const int32_t *order,
                              double *t_reached, double *t_c, double *mass, int32_t *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const InstState S = st[b];
    t_reached[b] = (double)S.step * desc[b].dt;
    t_c[b] = S.t_c;
    mass[b] = S.mass;
    int32_t s = S.status;
    const int err = ctl ? ctl->error : 0;
    if (err > 0 && order[err - 1] == b && s == kRunning) s = kTimeout;
    if (evolve_call && s == kRunning) {
        const long long n_end = (long long)ceil(t_end / desc[b].dt - 1e-9);
        if (S.step >= n_end) s = kDone;
    }
    status[b] = s;
}

}  // namespace adscl
