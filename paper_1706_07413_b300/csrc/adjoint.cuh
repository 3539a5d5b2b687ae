// adjoint.cuh -- discrete adjoint (reverse mode) of the evolution of evolve.cuh: the transpose of
// one RK4 step of the method-of-lines scheme of arXiv:1706.07413, Sec. II, including the
// constraint solve inside every stage, and the transpose of the sqrt(A)-weighted mode
// projection of spectrum.cuh.  Used for gradients of mode-energy functionals with respect to
// initial data.
//
// Work unit: one instance and checkpoint segment, on CL = 1 CTA (512 threads, 8 nodes per
// thread, the layout of evolve.cuh; N <= 4097) or on a CL = 2 thread-block cluster whose two
// CTAs own the two halves of the node blocks: 4 nodes per thread for N <= 4097, so that all
// 2 x 512 threads carry nodes (batches smaller than the SM count: each instance then occupies
// two SMs), 8 nodes per thread for 4097 < N <= 8193.
//   Phase F: from the segment's first slice, recompute its steps with the same discrete map as
//     evolve.cuh (affine-map scan for m, suffix sum for delta, table-driven exp) and store, for
//     every stage of every step, the stage input (Phi, Pi) and the stage's m, e^{-delta}, F and
//     alpha in HBM; nothing is recomputed later.
//   Phase B: run the steps backwards.  With lambda' the sensitivity to a step's output,
//     kbar_s = w_s dt lambda' + c_{s+1} dt ybar_{s+1},  ybar_s = R'(y_s)^T kbar_s,
//     lambda = lambda' + sum_s ybar_s,
//   where R'(y)^T applies, in this order: the transposed stencils of the right-hand side (gather
//   form on the ghost-extended index range, ghost values folded back onto the nodes they
//   mirror), the flux products, A = 1 - m K and F = A e^{-delta}, the m recurrence transposed
//   into a suffix affine scan mu_c = alpha_c mu_{c+1} + mbar_c, the delta suffix sum transposed
//   into a prefix sum, the derivatives of the per-cell RK4 maps (alpha, beta) and of the
//   Simpson increment, and the midpoint interpolation and rho = Phi^2 + Pi^2.
// Neighbour values go through global scratch arrays private to the CTA (cluster) and a barrier
// over the CTA (cluster: barrier.cluster with release / acquire semantics, which orders the global
// scratch accesses of both CTAs); the block scans carry the other rank's total through
// distributed shared memory.  The kernel is bound by FP64 issue, not by memory.  Instances are
// taken from an atomic counter by rank 0; no CTA waits on another outside its cluster.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "evolve.cuh"
#include "spectrum.cuh"

namespace adscl {

constexpr int kAP = 8;          // nodes per thread of a single-CTA instance
constexpr int kANT = 512;       // threads per CTA
constexpr int kANW = kANT / 32;
// kStageArrays (evolve.cuh): stored per stage: yP, yQ, M, E, F, AL
constexpr int kScrArrays = 21;   // CTA scratch arrays
// length of every scratch array: a compile-time stride (the adjoint's largest grid, 8193 points,
// rounded up), so that each array is the scratch base plus a constant and a thread's accesses
// are one base register plus immediate offsets
constexpr int kScrStride = 2 * kAP * kANT + 8;
// table t of the sweep's geometry block at index i (read-only path)
__device__ __forceinline__ double agv(const double *ag, int t, int i) { return __ldg(ag + t * kScrStride + i); }

// kAdjSegment: both phases of a segment; kAdjSegF / kAdjSegB: only the recomputation (phase F,
// from the checkpoint into the stage storage) or only the backward sweep (phase B, from the
// stage storage), so that the recomputation of one segment can run beside the sweep of the next
enum : int32_t { kAdjSegment = 0, kAdjSpectrum = 1, kAdjProject = 2, kAdjSegF = 3, kAdjSegB = 4 };

// The backward sweep's geometry (per grid size N <= 8193): kAgTables tables kScrStride doubles
// apart, so that one base pointer and immediate offsets reach all of them.  The first seven are
// copies of GeoTab's ws, wt, K, T, wsm3, wtm and iT12k; the others are scaled copies for the cell
// transpose: at the nodes 2 ws, 2 wt and 6 ws, at the cell midpoints 2 wsm3, 2 wtm and (8/3) wsm3.
// With them the transpose forms twice the node and midpoint sensitivities of rho directly (the
// factor 2 of d rho = 2 Phi dPhi + 2 Pi dPi) and the forward quantities y2 = 1/3 - ws rho and
// ca = 2 - 6 ws rho in one FMA each.
enum : int {
    kAgWs = 0, kAgWt, kAgK, kAgT, kAgWsm3, kAgWtm, kAgIT12k,
    kAgWs2, kAgWt2, kAgWs6, kAgWsm3x2, kAgWtm2, kAgWsm3x83, kAgTables
};

struct AdjArgs {
    const InstDesc *desc;
    const GeoTab *geo;
    const double *const *ageo;   // per grid size: the sweep's geometry block (null for N > 8193)
    const EigTab *eig;
    const double *exptab;
    const int32_t *order;
    int32_t nwork;
    int32_t *queue;
    int32_t mode;
    // segment mode
    const double *ckP, *ckQ;  // packed slices at the segment start
    double *outP, *outQ;      // phase F: packed slices receiving the segment's last slice (or null)
    int32_t nsteps;           // steps of this segment
    double *stage;            // per instance: nsteps_cap * 4 stages * kStageArrays * Nmax (the
                              // layout of the evolution kernel's stage record, stage_slot)
    int32_t nsteps_cap;
    double *lamP, *lamQ;      // packed adjoint state, updated in place
    double *scratch;          // per CTA (cluster): kScrArrays * kScrStride
    int32_t Nmax;
    // spectrum mode: lambda += d(sum_j Ebar_j E_j)/d(slice)
    const double *Ebar;       // B x J
    int32_t J;
    const double *sP, *sQ;    // packed slice
    // projection mode: dJda[b, j] = sum_{i < N-1} lamQ_i e_j(x_i), j < J
    double *dJda;
};

// value at index i in [-8, N+7] with the parity rule (u_{-k} = p0 u_k, u_{N-1+k} = p1 u_{N-1-k})
__device__ __forceinline__ double gv(const double *u, int N, int i, double p0, double p1) {
    if (i < 0) return p0 * u[-i];
    if (i > N - 1) return p1 * u[2 * (N - 1) - i];
    return u[i];
}
// value of a row-restricted array on the extended range (zero outside [0, N-1])
__device__ __forceinline__ double rv(const double *v, int N, int i) {
    return (i < 0 || i > N - 1) ? 0.0 : v[i];
}
// the same for a thread whose reads all lie inside the grid (INT): a plain load, no range tests
template <bool INT>
__device__ __forceinline__ double gvi(const double *u, int N, int i, double p0, double p1) {
    if constexpr (INT) return u[i]; else return gv(u, N, i, p0, p1);
}
template <bool INT>
__device__ __forceinline__ double rvi(const double *v, int N, int i) {
    if constexpr (INT) return v[i]; else return rv(v, N, i);
}
// every node this thread reads in the transposed stencils and cell maps (its AP nodes and three
// on each side, ghost folds included) is an interior node
template <int AP>
__device__ __forceinline__ bool reads_interior(int i0, int N) { return i0 >= 4 && i0 + AP + 4 <= N - 1; }

// ------------------------------------------------------------------ block scans (512 threads)
// The affine scans and the sums use disjoint slots (a, b, c, e, pb and d, f, pd), so a sum may
// follow an affine scan without a barrier between them; a scan's slots are written again only by
// the next scan of its kind, which every call site separates from this one by barriers.
struct ScanShared {
    double a[kANW], b[kANW], c[kANW], d[kANW], e[kANW], f[kANW];
    double pa, pb, pd;   // total of the other rank of a 2-CTA cluster (written by it)
};

// node ownership of this thread for grid size N: rank r of a CL-CTA cluster owns node blocks
// ceil(r T / CL) .. ceil((r+1) T / CL) - 1 of the T blocks of AP nodes
struct Own {
    int T, i0;
    bool act, last;
};
template <int CL, int AP>
__device__ __forceinline__ Own own_of(int N)
{
    Own o;
    o.T = (N - 1) / AP;
    const int rank = (CL > 1) ? cluster_rank() : 0;
    const int bs = (rank * o.T + CL - 1) / CL, be = ((rank + 1) * o.T + CL - 1) / CL;
    const int t = bs + (int)threadIdx.x;
    o.i0 = t * AP;
    o.act = t < be;
    o.last = t == o.T - 1;
    return o;
}

// An affine scan and a sum scan in one pass with one CTA barrier and one cluster barrier, over
// the threads of both ranks of a 2-CTA cluster.  The affine maps x -> a x + b compose in thread
// order and the scan returns the b part of the exclusive composition applied to 0; the sums are
// exclusive.  kAffSuffix = false: the affine prefix (threads ascending, rank 0's threads first)
// and the suffix sum; kAffSuffix = true: the affine suffix (threads descending, rank 1's threads
// first; the thread's map is x_left = a x_right + b) and the prefix sum.
template <int CL, bool kAffSuffix>
__device__ void scan_pair(double a, double b, double x, ScanShared &sh, double &raff, double &rsum)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (kAffSuffix) {
            const double an = __shfl_down_sync(FULL, a, o), bn = __shfl_down_sync(FULL, b, o);
            const double xn = __shfl_up_sync(FULL, x, o);
            if (lane + o < 32) { b = fma(a, bn, b); a = mul_f(a, an); }
            if (lane >= o) x = add_f(x, xn);
        } else {
            const double ap = __shfl_up_sync(FULL, a, o), bp = __shfl_up_sync(FULL, b, o);
            const double xp = __shfl_down_sync(FULL, x, o);
            if (lane >= o) { b = fma(a, bp, b); a = mul_f(a, ap); }
            if (lane + o < 32) x = add_f(x, xp);
        }
    }
    double aEx, bEx, ex;
    if (kAffSuffix) {
        aEx = __shfl_down_sync(FULL, a, 1);
        bEx = __shfl_down_sync(FULL, b, 1);
        ex = __shfl_up_sync(FULL, x, 1);
        if (lane == 31) { aEx = 1.0; bEx = 0.0; }
        if (lane == 0) { ex = 0.0; sh.a[wid] = a; sh.b[wid] = b; }
        if (lane == 31) sh.d[wid] = x;
    } else {
        aEx = __shfl_up_sync(FULL, a, 1);
        bEx = __shfl_up_sync(FULL, b, 1);
        ex = __shfl_down_sync(FULL, x, 1);
        if (lane == 0) { aEx = 1.0; bEx = 0.0; sh.d[wid] = x; }
        if (lane == 31) { ex = 0.0; sh.a[wid] = a; sh.b[wid] = b; }
    }
    __syncthreads();
    if (wid == 0) {
        double A = lane < kANW ? sh.a[lane] : 1.0, B = lane < kANW ? sh.b[lane] : 0.0;
        double X = lane < kANW ? sh.d[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < kANW; o <<= 1) {
            if (kAffSuffix) {
                const double an = __shfl_down_sync(FULL, A, o), bn = __shfl_down_sync(FULL, B, o);
                const double xn = __shfl_up_sync(FULL, X, o);
                if (lane + o < kANW) { B = fma(A, bn, B); A = mul_f(A, an); }
                if (lane >= o) X = add_f(X, xn);
            } else {
                const double ap = __shfl_up_sync(FULL, A, o), bp = __shfl_up_sync(FULL, B, o);
                const double xp = __shfl_down_sync(FULL, X, o);
                if (lane >= o) { B = fma(A, bp, B); A = mul_f(A, ap); }
                if (lane + o < kANW) X = add_f(X, xp);
            }
        }
        double bw, aw, w;
        if (kAffSuffix) {
            bw = __shfl_down_sync(FULL, B, 1);
            aw = __shfl_down_sync(FULL, A, 1);
            w = __shfl_up_sync(FULL, X, 1);
            if (lane + 1 >= kANW) { bw = 0.0; aw = 1.0; }
            if (lane == 0) w = 0.0;
        } else {
            bw = __shfl_up_sync(FULL, B, 1);
            aw = __shfl_up_sync(FULL, A, 1);
            w = __shfl_down_sync(FULL, X, 1);
            if (lane == 0) { bw = 0.0; aw = 1.0; }
            if (lane + 1 >= kANW) w = 0.0;
        }
        if (lane < kANW) { sh.c[lane] = bw; sh.e[lane] = aw; sh.f[lane] = w; }
        if constexpr (CL == 2) {
            const int rk = cluster_rank();
            if (kAffSuffix) {   // rank 1's total map to rank 0, rank 0's sum to rank 1
                if (lane == 0 && rk == 1) st_peer(&sh.pb, B, 0);
                if (lane == kANW - 1 && rk == 0) st_peer(&sh.pd, X, 1);
            } else {            // rank 0's total map to rank 1, rank 1's sum to rank 0
                if (lane == kANW - 1 && rk == 0) st_peer(&sh.pb, B, 1);
                if (lane == 0 && rk == 1) st_peer(&sh.pd, X, 0);
            }
        }
    }
    csync<CL>();
    raff = fma(aEx, sh.c[wid], bEx);
    rsum = add_f(ex, sh.f[wid]);
    if constexpr (CL == 2) {
        const int rk = cluster_rank();
        if (rk == (kAffSuffix ? 0 : 1)) raff = fma(mul_f(aEx, sh.e[wid]), sh.pb, raff);   // the other rank's maps first
        if (rk == (kAffSuffix ? 1 : 0)) rsum = add_f(rsum, sh.pd);
    }
}

// ------------------------------------------------------------------ per-cell RK4 map of m
// The map in the form of the evolution kernel: with q = h b / 6, r = h a / 6 at the cell's left
// end (q0, r0), midpoint (qm, tm; qm3 = 3 qm) and right end (q1, r1),
//   y2 = 1/3 - q0, y3 = 1/3 - qm3 y2, ca = 2 - 6 q1, e = 2 - qm3 ca, w2 = tm - qm3 r0,
//   alpha = (y2 - q1) + y3 e,  beta = (r0 + r1) + ca tm + e w2,  Delta = q0 + q1 + (4/3) qm3.
struct CellFwd {
    double qn0, qn1, rn0, rn1, p16, q16, qm3, tm, y2, y3, ca, e, w2, al, be, De;
};

// forward cell data of cell c from Phi, Pi at nodes c-1 .. c+2 (ghosts by parity) and the node
// factors q = ws rho, r = wt rho at its two ends
__device__ __forceinline__ CellFwd cell_fwd_n(double qn0, double rn0, double qn1, double rn1, double pm1,
                                             double p0, double p1, double p2, double qm1, double q0,
                                             double q1, double q2, const GeoTab &g, int c)
{
    CellFwd r;
    r.qn0 = qn0;
    r.rn0 = rn0;
    r.qn1 = qn1;
    r.rn1 = rn1;
    r.p16 = fma(9.0, add_f(p0, p1), -add_f(pm1, p2));
    r.q16 = fma(9.0, add_f(q0, q1), -add_f(qm1, q2));
    const double rm = fma(r.p16, r.p16, mul_f(r.q16, r.q16));
    r.qm3 = mul_f(__ldg(g.wsm3 + c), rm);
    r.tm = mul_f(__ldg(g.wtm + c), rm);
    r.De = fma(4.0 / 3.0, r.qm3, add_f(r.qn0, r.qn1));
    r.y2 = add_f(-r.qn0, 1.0 / 3.0);
    r.y3 = fma(-r.qm3, r.y2, 1.0 / 3.0);
    r.ca = fma(-6.0, r.qn1, 2.0);
    r.e = fma(-r.qm3, r.ca, 2.0);
    r.al = fma(r.y3, r.e, add_f(r.y2, -r.qn1));
    r.w2 = fma(-r.qm3, r.rn0, r.tm);
    r.be = fma(r.e, r.w2, fma(r.ca, r.tm, add_f(r.rn0, r.rn1)));
    return r;
}

// ------------------------------------------------------------------ CTA scratch layout
struct Scr {
    double *uP, *uQ;     // current slice u_n (phase F)
    double *aP, *aQ;     // RK4 accumulator (phase F)
    double *f, *u;       // fluxes F Pi, tan^2 F Phi (phase F)
    double *vP, *vQ;     // kbar restricted to rows (phase B)
    double *fb, *ub;     // fbar, ubar on nodes (phase B)
    double *r1, *pb, *qb;  // per cell: rho_bar of its right node, p16_bar, q16_bar
    double *lo, *lq;     // lambda' (sensitivity to the step output)
    double *ybP, *ybQ;   // ybar of the previous (later) stage
    double *mb;          // mbar, then mu
    double *dlb;         // delta_bar
    double *v2;          // iT12 kbar_Pi (phase B: the Pi-dot sensitivities seen by the u stencil)
};

__device__ __forceinline__ Scr scratch_of(double *base)
{
    constexpr int L = kScrStride;
    Scr s;
    s.uP = base; s.uQ = base + L; s.aP = base + 2 * L; s.aQ = base + 3 * L;
    s.f = base + 4 * L; s.u = base + 5 * L; s.vP = base + 6 * L; s.vQ = base + 7 * L;
    s.fb = base + 8 * L; s.ub = base + 9 * L; s.r1 = base + 10 * L; s.pb = base + 11 * L;
    s.qb = base + 12 * L; s.lo = base + 13 * L; s.lq = base + 14 * L; s.ybP = base + 15 * L;
    s.ybQ = base + 16 * L; s.mb = base + 17 * L; s.dlb = base + 18 * L; s.v2 = base + 19 * L;
    return s;
}

// ------------------------------------------------------------------ stage forward
// Constraint solve on the stage slice (yP, yQ) (node N-1 and all nodes written, zero at N-1);
// stores M, E = e^{-delta}, F = A E on nodes and AL = alpha on cells; computes the fluxes into
// scr.f, scr.u and, if kP != nullptr, the stage derivative (kP, kQ) on the thread's nodes.
template <int CL, int AP>
__device__ void stage_forward(const double *yP, const double *yQ, double *M, double *E, double *F, double *AL,
                              const Scr &scr, double *kP, double *kQ, const InstDesc &d, const GeoTab &g,
                              const double *tab, ScanShared &sh, bool with_rhs)
{
    const int N = d.N;
    const Own o = own_of<CL, AP>(N);
    const bool act = o.act, last = o.last;
    const int i0 = o.i0;
    double De[AP], al[AP], be[AP];
    double aT = 1.0, bT = 0.0, SD = 0.0;
    if (act) {
        // the cell maps with the node quantities carried from cell to cell, compiled with plain
        // loads for warps whose threads read only interior nodes and with the parity ghosts
        auto cells = [&](auto interior) {
        constexpr bool INT = decltype(interior)::value;
        double pm1 = gvi<INT>(yP, N, i0 - 1, -1.0, 1.0), p0 = yP[i0], p1 = yP[i0 + 1];
        double qm1 = gvi<INT>(yQ, N, i0 - 1, 1.0, -1.0), q0 = yQ[i0], q1 = yQ[i0 + 1];
        const double rho0 = fma(p0, p0, mul_f(q0, q0));
        double qn0 = mul_f(__ldg(g.ws + i0), rho0), rn0 = mul_f(__ldg(g.wt + i0), rho0);
#pragma unroll
        for (int k = 0; k < AP; ++k) {
            const int c = i0 + k;
            const double p2 = gvi<INT>(yP, N, c + 2, -1.0, 1.0), q2 = gvi<INT>(yQ, N, c + 2, 1.0, -1.0);
            const double rho1 = fma(p1, p1, mul_f(q1, q1));
            const double qn1 = mul_f(__ldg(g.ws + c + 1), rho1), rn1 = mul_f(__ldg(g.wt + c + 1), rho1);
            const CellFwd cf = cell_fwd_n(qn0, rn0, qn1, rn1, pm1, p0, p1, p2, qm1, q0, q1, q2, g, c);
            pm1 = p0; p0 = p1; p1 = p2;
            qm1 = q0; q0 = q1; q1 = q2;
            qn0 = qn1; rn0 = rn1;
            De[k] = cf.De;
            al[k] = cf.al;
            be[k] = cf.be;
            AL[c] = cf.al;
            if (k == 0) { aT = cf.al; bT = cf.be; SD = cf.De; }
            else { bT = fma(cf.al, bT, cf.be); aT = mul_f(aT, cf.al); SD = add_f(SD, cf.De); }
        }
        };
        if (__all_sync(__activemask(), reads_interior<AP>(i0, N))) cells(std::true_type{});
        else cells(std::false_type{});
    }
    double mstart, dend;   // m at node i0; the sum of Delta over the cells from node i0 + AP on
    scan_pair<CL, false>(aT, bT, SD, sh, mstart, dend);
    double g1 = 0.0, g2 = 0.0, um1 = 0.0, um2 = 0.0;
    if (act) {
        double dc = dend;
#pragma unroll
        for (int k = AP - 1; k >= 0; --k) { dc = add_f(dc, De[k]); De[k] = dc; }
        double m = mstart;
#pragma unroll
        for (int k = 0; k < AP; ++k) {
            const int i = i0 + k;
            const double A = fma(-m, __ldg(g.K + i), 1.0);
            const double Ei = a_exp_neg(1.0, De[k], tab);
            const double Fi = mul_f(A, Ei);
            M[i] = m;
            E[i] = Ei;
            F[i] = Fi;
            const double gi = mul_f(Fi, yP[i]);
            const double ui = mul_f(__ldg(g.T + i), gi);
            scr.f[i] = mul_f(Fi, yQ[i]);
            scr.u[i] = ui;
            if (k == 1) g1 = gi;
            if (k == 2) g2 = gi;
            if (k == AP - 1) um1 = ui;
            if (k == AP - 2) um2 = ui;
            m = fma(al[k], m, be[k]);
        }
        if (last) {   // the last thread owns nodes N-3 and N-2 (AP >= 2)
            M[N - 1] = m;
            E[N - 1] = 1.0;
            F[N - 1] = 1.0;
            scr.f[N - 1] = 0.0;
            scr.u[N - 1] = (4.0 * um1 - um2) * (1.0 / 3.0);   // u(pi/2) by even extrapolation
        }
    }
    csync<CL>();
    if (!with_rhs || !act) return;
    // the stage derivative, compiled with and without range tests as the cell maps
    auto rhs = [&](auto interior) {
    constexpr bool INT = decltype(interior)::value;
#pragma unroll
    for (int k = 0; k < AP; ++k) {
        const int i = i0 + k;
        const double Df = fma(8.0, add_f(gvi<INT>(scr.f, N, i + 1, 1.0, -1.0), -gvi<INT>(scr.f, N, i - 1, 1.0, -1.0)),
                              add_f(gvi<INT>(scr.f, N, i - 2, 1.0, -1.0), -gvi<INT>(scr.f, N, i + 2, 1.0, -1.0)));
        const double Du = fma(8.0, add_f(gvi<INT>(scr.u, N, i + 1, -1.0, 1.0), -gvi<INT>(scr.u, N, i - 1, -1.0, 1.0)),
                              add_f(gvi<INT>(scr.u, N, i - 2, -1.0, 1.0), -gvi<INT>(scr.u, N, i + 2, -1.0, 1.0)));
        const double kp = fma(-20.0, yP[i], fma(15.0, add_f(gvi<INT>(yP, N, i - 1, -1, 1), gvi<INT>(yP, N, i + 1, -1, 1)),
                          fma(-6.0, add_f(gvi<INT>(yP, N, i - 2, -1, 1), gvi<INT>(yP, N, i + 2, -1, 1)),
                              add_f(gvi<INT>(yP, N, i - 3, -1, 1), gvi<INT>(yP, N, i + 3, -1, 1)))));
        const double kq = fma(-20.0, yQ[i], fma(15.0, add_f(gvi<INT>(yQ, N, i - 1, 1, -1), gvi<INT>(yQ, N, i + 1, 1, -1)),
                          fma(-6.0, add_f(gvi<INT>(yQ, N, i - 2, 1, -1), gvi<INT>(yQ, N, i + 2, 1, -1)),
                              add_f(gvi<INT>(yQ, N, i - 3, 1, -1), gvi<INT>(yQ, N, i + 3, 1, -1)))));
        double dP = fma(d.c12, Df, mul_f(d.cko, kp));
        double dQ = fma(__ldg(g.iT12 + i), Du, mul_f(d.cko, kq));
        if (!INT && i == 0) {
            dP = 0.0;
            dQ = fma(d.c3, fma(16.0, g1, -2.0 * g2), d.cko * kq);
        }
        kP[i] = dP;
        kQ[i] = dQ;
    }
    };
    if (__all_sync(__activemask(), reads_interior<AP>(i0, N))) rhs(std::true_type{});
    else rhs(std::false_type{});
}

// ------------------------------------------------------------------ constraint transpose
// Given Abar-derived mbar (scr.mb, nodes) and delta_bar (scr.dlb, nodes), accumulate into
// (yb P, yb Q) += d/d(yP, yQ) on the thread's nodes.
template <int CL, int AP>
__device__ void constraint_backward(const double *yP, const double *yQ, const double *M, const double *AL,
                                    const Scr &scr, double *ybP, double *ybQ, const InstDesc &d,
                                    const double *ag, ScanShared &sh)
{
    const int N = d.N;
    const Own o = own_of<CL, AP>(N);
    const bool act = o.act;
    const int i0 = o.i0;
    // mu_c = alpha_c mu_{c+1} + mbar_c, mu_{N-1} = 0: suffix affine scan
    double aT = 1.0, bT = 0.0, SP = 0.0;
    if (act) {   // seeded with the last cell's map and the first node's value
        aT = AL[i0 + AP - 1];
        bT = scr.mb[i0 + AP - 1];
#pragma unroll
        for (int k = AP - 2; k >= 0; --k) {
            const int c = i0 + k;
            const double a = AL[c];
            bT = fma(a, bT, scr.mb[c]);
            aT = mul_f(aT, a);
        }
        SP = scr.dlb[i0];
#pragma unroll
        for (int k = 1; k < AP; ++k) SP = add_f(SP, scr.dlb[i0 + k]);
    }
    double mu_end, dpre;   // mu at node i0 + AP; the sum of delta_bar over the nodes < i0
    scan_pair<CL, true>(aT, bT, SP, sh, mu_end, dpre);
    if (act) {
        double mu = mu_end;
        double mun[AP];   // mu at node c+1 for each own cell
#pragma unroll
        for (int k = AP - 1; k >= 0; --k) {
            mun[k] = mu;
            mu = fma(AL[i0 + k], mu, scr.mb[i0 + k]);
        }
        double Db = dpre;
        double n0s[AP];
        // the cell loop, compiled once with plain loads (warps whose threads read only interior
        // nodes: all but the two at the ends of the grid) and once with the parity ghosts.
        // Per cell c: the forward quantities of the m map (the linearisation point; rho and the
        // node factor r carried from cell to cell), then the transpose of
        //   alpha = (y2 - q1) + y3 e,  beta = (r0 + r1) + ca tm + e w2,  Delta = q0 + q1 + (4/3) qm3
        // with y2 = 1/3 - q0, y3 = 1/3 - qm3 y2, ca = 2 - 6 q1, e = 2 - qm3 ca, w2 = tm - qm3 r0,
        // at alpha_bar = mu m_c, beta_bar = mu (mu = mu_{c+1}), Delta_bar = Db.  Its partial
        // derivatives give, with u = 1 - e qm3:
        //   r0_bar = mu u,  q0_bar = Db - mu m_c u,  r1_bar = mu,  tm_bar = mu (ca + e),
        //   q1_bar = mu (m_c (6 qm3 y3 - 1) + 6 (qm3 w2 - tm)) + Db,
        //   qm3_bar = (4/3) Db - mu (m_c (e y2 + y3 ca) + (w2 ca + e r0)),
        // and, through q = ws rho, r = wt rho at the nodes and qm3 = wsm3 rm, tm = wtm rm at the
        // midpoint, twice the rho sensitivities:
        //   2 rho_bar(node c) = mu u (2 wt - 2 ws m_c) + 2 ws Db  (cell c's left node),
        //   2 rho_bar(node c+1) = 2 ws q1_bar + 2 wt mu          (its right node),
        //   2 rm_bar = mu (2 wtm (ca + e) - 2 wsm3 (...)) + (8/3) wsm3 Db.
        auto cells = [&](auto interior) {
        constexpr bool INT = decltype(interior)::value;
        double pm1 = gvi<INT>(yP, N, i0 - 1, -1.0, 1.0), p0 = yP[i0], p1 = yP[i0 + 1];
        double qm1 = gvi<INT>(yQ, N, i0 - 1, 1.0, -1.0), q0 = yQ[i0], q1 = yQ[i0 + 1];
        double rho0 = fma(p0, p0, mul_f(q0, q0));
        double r0 = mul_f(agv(ag, kAgWt, i0), rho0);
#pragma unroll
        for (int k = 0; k < AP; ++k) {
            const int c = i0 + k;
            Db = add_f(Db, scr.dlb[c]);               // Delta_bar_c = sum_{i <= c} delta_bar_i
            const double p2 = gvi<INT>(yP, N, c + 2, -1.0, 1.0), q2 = gvi<INT>(yQ, N, c + 2, 1.0, -1.0);
            const double rho1 = fma(p1, p1, mul_f(q1, q1));
            const double y2 = fma(-agv(ag, kAgWs, c), rho0, 1.0 / 3.0);
            const double ca = fma(-agv(ag, kAgWs6, c + 1), rho1, 2.0);
            const double p16 = fma(9.0, add_f(p0, p1), -add_f(pm1, p2));
            const double q16 = fma(9.0, add_f(q0, q1), -add_f(qm1, q2));
            const double rm = fma(p16, p16, mul_f(q16, q16));
            const double qm3 = mul_f(agv(ag, kAgWsm3, c), rm);
            const double tm = mul_f(agv(ag, kAgWtm, c), rm);
            const double y3 = fma(-qm3, y2, 1.0 / 3.0);
            const double e = fma(-qm3, ca, 2.0);
            const double w2 = fma(-qm3, r0, tm);
            const double r1 = mul_f(agv(ag, kAgWt, c + 1), rho1);
            const double mc = mun[k], m = M[c];
            const double u = fma(-e, qm3, 1.0);
            n0s[k] = fma(mul_f(mc, u), fma(-agv(ag, kAgWs2, c), m, agv(ag, kAgWt2, c)), mul_f(agv(ag, kAgWs2, c), Db));
            const double q6 = mul_f(6.0, qm3);
            const double q1b = fma(mc, fma(m, fma(q6, y3, -1.0), fma(q6, w2, mul_f(-6.0, tm))), Db);
            scr.r1[c] = fma(agv(ag, kAgWs2, c + 1), q1b, mul_f(agv(ag, kAgWt2, c + 1), mc));
            const double inner = fma(m, fma(e, y2, mul_f(y3, ca)), fma(w2, ca, mul_f(e, r0)));
            const double X = fma(-agv(ag, kAgWsm3x2, c), inner, mul_f(agv(ag, kAgWtm2, c), add_f(ca, e)));
            const double rmb2 = fma(mc, X, mul_f(agv(ag, kAgWsm3x83, c), Db));   // 2 rm_bar
            // rho_m = (p16^2 + q16^2) / 256, the 1/256 folded into wsm3 and wtm
            scr.pb[c] = mul_f(p16, rmb2);
            scr.qb[c] = mul_f(q16, rmb2);
            pm1 = p0; p0 = p1; p1 = p2;
            qm1 = q0; q0 = q1; q1 = q2;
            rho0 = rho1; r0 = r1;
        }
        };
        if (__all_sync(__activemask(), reads_interior<AP>(i0, N))) cells(std::true_type{});
        else cells(std::false_type{});
        // keep the node parts in the scratch f/u slots (free in phase B)
#pragma unroll
        for (int k = 0; k < AP; ++k) scr.fb[i0 + k] = n0s[k];
    }
    csync<CL>();
    if (act) {
        // compiled with and without range tests, as the cell loop
        auto nodes = [&](auto interior) {
        constexpr bool INT = decltype(interior)::value;
#pragma unroll
        for (int k = 0; k < AP; ++k) {
            const int j = i0 + k;
            // twice rho_bar at node j: the left-node part of cell j and the right-node part of cell j-1
            const double rb = add_f(scr.fb[j], (INT || j >= 1) ? scr.r1[j - 1] : 0.0);
            // transpose of p16_c = 9 (w_c + w_{c+1}) - (w_{c-1} + w_{c+2}), cells 0 .. N-2
            auto itp = [&](const double *b, int x) {
                return fma(9.0, add_f(rvi<INT>(b, N - 1, x), rvi<INT>(b, N - 1, x - 1)),
                           -add_f(rvi<INT>(b, N - 1, x + 1), rvi<INT>(b, N - 1, x - 2)));
            };
            double pP = itp(scr.pb, j), pQ = itp(scr.qb, j);
            if constexpr (!INT) {
                if (j == 1) { pP += -itp(scr.pb, -1); pQ += itp(scr.qb, -1); }                // ghost -1
                if (j == N - 2) { pP += itp(scr.pb, N); pQ += -itp(scr.qb, N); }              // ghost N
            }
            ybP[j] = add_f(ybP[j], fma(yP[j], rb, pP));   // d rho = 2 Phi dPhi + 2 Pi dPi
            ybQ[j] = add_f(ybQ[j], fma(yQ[j], rb, pQ));
        }
        };
        if (__all_sync(__activemask(), reads_interior<AP>(i0, N))) nodes(std::true_type{});
        else nodes(std::false_type{});
    }
    // no barrier here: every caller updates only its own nodes next and then synchronises
    // before scr.pb, qb, r1, fb are written again
}

// ------------------------------------------------------------------ stage backward
// ybar = R'(y)^T kbar with kbar in (scr.vP, scr.vQ) (already restricted to rows, and scaled by
// c12 = 1/(12 h) and cq, the factors of Phi-dot and Pi-dot), written to (ybP, ybQ) (overwritten)
// on the thread's nodes.
template <int CL, int AP>
__device__ void stage_backward(const double *yP, const double *yQ, const double *M, const double *E,
                               const double *F, const double *AL, const Scr &scr, double *ybP, double *ybQ,
                               const InstDesc &d, const double *ag, ScanShared &sh)
{
    const int N = d.N;
    const Own o = own_of<CL, AP>(N);
    const bool act = o.act, last = o.last;
    const int i0 = o.i0;
    const double *vP = scr.vP, *vQ = scr.vQ;
    const double *v2 = scr.v2;   // iT12-weighted Pi-dot sensitivities (zero at rows 0 and N-1)
    if (act) {
        const double vQ0 = vQ[0];
        // the node loop, compiled once with plain loads (warps whose threads read only interior
        // nodes) and once with the range tests and the ghost folds of the grid's two ends
        auto nodes = [&](auto interior) {
        constexpr bool INT = decltype(interior)::value;
        auto Dr = [&](const double *v, int x) {   // raw 4th-order difference of a row-restricted array
            return fma(8.0, add_f(rvi<INT>(v, N, x + 1), -rvi<INT>(v, N, x - 1)),
                       add_f(rvi<INT>(v, N, x - 2), -rvi<INT>(v, N, x + 2)));
        };
        auto KOr = [&](const double *v, int x) {  // raw dissipation stencil of a row-restricted array
            return fma(-20.0, rvi<INT>(v, N, x), fma(15.0, add_f(rvi<INT>(v, N, x - 1), rvi<INT>(v, N, x + 1)),
                   fma(-6.0, add_f(rvi<INT>(v, N, x - 2), rvi<INT>(v, N, x + 2)),
                       add_f(rvi<INT>(v, N, x - 3), rvi<INT>(v, N, x + 3)))));
        };
#pragma unroll
        for (int k = 0; k < AP; ++k) {
            const int j = i0 + k;
            // transposed stencils on the extended range, ghosts folded back (parities:
            // f even/odd, u odd/even, Phi odd/even, Pi even/odd about 0 / pi/2)
            double fbx = -Dr(vP, j), ubx = -Dr(v2, j), kpx = KOr(vP, j), kqx = KOr(vQ, j);
            if constexpr (!INT) {
                if (j >= 1 && j <= 3) {
                    fbx += -Dr(vP, -j);
                    ubx -= -Dr(v2, -j);
                    kpx -= KOr(vP, -j);
                    kqx += KOr(vQ, -j);
                }
                if (j >= N - 4 && j <= N - 2) {
                    const int x = 2 * (N - 1) - j;
                    fbx -= -Dr(vP, x);
                    ubx += -Dr(v2, x);
                    kpx += KOr(vP, x);
                    kqx -= KOr(vQ, x);
                }
                if (j == N - 2) ubx += (4.0 / 3.0) * (-Dr(v2, N - 1));   // u(pi/2) extrapolation
                if (j == N - 3) ubx += (-1.0 / 3.0) * (-Dr(v2, N - 1));
            }
            const double fb = fbx;   // (vP carries the factor c12, vQ the factor cq)
            double gb = mul_f(agv(ag, kAgT, j), ubx);
            if constexpr (!INT) {
                if (j == 1) gb = fma(16.0 * d.c3q, vQ0, gb);            // Pi-dot(0) = 3 (F Phi)'(0)
                if (j == 2) gb = fma(-2.0 * d.c3q, vQ0, gb);
            }
            const double Fj = F[j];
            const double Fb = fma(fb, yQ[j], mul_f(gb, yP[j]));
            ybQ[j] = fma(fb, Fj, d.ko ? kqx : 0.0);
            ybP[j] = fma(gb, Fj, mul_f(d.rko, kpx));
            const double Ab = mul_f(Fb, E[j]);
            scr.dlb[j] = mul_f(-Fb, Fj);
            scr.mb[j] = mul_f(-Ab, agv(ag, kAgK, j));
        }
        };
        if (__all_sync(__activemask(), reads_interior<AP>(i0, N))) nodes(std::true_type{});
        else nodes(std::false_type{});
        if (last) { scr.dlb[N - 1] = 0.0; scr.mb[N - 1] = 0.0; }
    }
    // no barrier: the constraint transpose reads only this thread's mb, dlb before its scans'
    // barriers, and vP, vQ, v2 are written again only after the next stage's first barrier
    constraint_backward<CL, AP>(yP, yQ, M, AL, scr, ybP, ybQ, d, ag, sh);
}

// ------------------------------------------------------------------ the kernel
// AP nodes per thread: (CL, AP) = (1, 8) and (2, 4) for N <= 4097 (on a 2-CTA cluster every
// thread of both CTAs carries nodes), (2, 8) for N <= 8193.  SWEEP = true compiles the backward
// sweep alone (mode kAdjSegB only): its registers are then allocated for that path, not for the
// longest-lived values of the recomputation and the spectrum transpose.
template <int CL, int AP, bool SWEEP>
__global__ void __launch_bounds__(kANT, 1) adjoint_kernel(AdjArgs a)
{
    static_assert(CL == 1 || CL == 2, "one CTA or a 2-CTA cluster per instance");
    __shared__ ScanShared sh;
    __shared__ double s_tab[kExpTableSize];
    __shared__ int s_item;
    // phase B's factors of stage s for the current work item: w_s dt c12, w_s dt cq, c_{s+1} dt c12,
    // c_{s+1} dt cq (computed once per work item instead of by every thread in every stage)
    __shared__ double s_kc[4][4];
    const int tid = threadIdx.x;
    const int rank = (CL > 1) ? cluster_rank() : 0;
    if constexpr (!SWEEP)   // the exponential is evaluated only in the forward stages
        for (int i = tid; i < kExpTableSize; i += kANT) s_tab[i] = a.exptab[i];
    csync<CL>();   // every CTA of the cluster has started before any remote shared-memory store
    // one scratch region per CTA (CL = 1) or per cluster (CL = 2: shared by both ranks)
    const Scr scr = scratch_of(a.scratch + (size_t)(blockIdx.x / CL) * kScrArrays * kScrStride);
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    const double wst[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

    for (;;) {
        if (tid == 0 && rank == 0) {
            const int v = atomicAdd(a.queue, 1);
            s_item = v;
            if constexpr (CL == 2) st_peer(&s_item, v, 1);
        }
        csync<CL>();
        const int q = s_item;
        if (tid == 0 && q < a.nwork) {
            const InstDesc dq = a.desc[a.order[q]];
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                s_kc[st][0] = wst[st] * dq.dtc;
                s_kc[st][1] = wst[st] * dq.dtq;
                s_kc[st][2] = st < 3 ? cst[st + 1] * dq.dtc : 0.0;
                s_kc[st][3] = st < 3 ? cst[st + 1] * dq.dtq : 0.0;
            }
        }
        csync<CL>();   // also publishes s_kc (its previous readers passed the barrier above)
        if (q >= a.nwork) break;
        const int b = a.order[q];
        const InstDesc d = a.desc[b];
        const GeoTab g = a.geo[d.geo];
        const double *ag = a.ageo[d.geo];
        const int N = d.N;
        const Own own = own_of<CL, AP>(N);
        const bool act = own.act;
        const int i0 = own.i0;
        double *lamP = a.lamP + d.off, *lamQ = a.lamQ + d.off;

        if (!SWEEP && a.mode == kAdjProject) {
            if (rank == 0) {
                const EigTab t = a.eig[d.geo];
                const int lane = tid & 31, warp = tid >> 5;
                for (int j = warp; j < a.J; j += kANW) {
                    double s = 0.0;
                    for (int i = lane; i < N - 1; i += 32) s = fma(lamQ[i], __ldg(t.e + (size_t)j * N + i), s);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) a.dJda[(size_t)b * a.J + j] = s;
                }
            }
            csync<CL>();
            continue;
        }

        // per-stage storage of this work item
        const size_t stN = (size_t)a.Nmax;
        double *stage_base = a.stage + (size_t)b * a.nsteps_cap * 4 * kStageArrays * stN;
        auto slot = [&](int n, int s, int arr) { return stage_base + (((size_t)n * 4 + s) * kStageArrays + arr) * stN; };

        if (!SWEEP && a.mode == kAdjSpectrum) {
            // constraint solve of the slice, projections, then the transpose into lambda
            const double *sP = a.sP + d.off, *sQ = a.sQ + d.off;
            double *yP = slot(0, 0, 0), *yQ = slot(0, 0, 1), *M = slot(0, 0, 2), *E = slot(0, 0, 3),
                   *F = slot(0, 0, 4), *AL = slot(0, 0, 5);
            if (act) {
#pragma unroll
                for (int k = 0; k < AP; ++k) { yP[i0 + k] = sP[i0 + k]; yQ[i0 + k] = sQ[i0 + k]; }
                if (own.last) { yP[N - 1] = 0.0; yQ[N - 1] = 0.0; }
            }
            csync<CL>();
            stage_forward<CL, AP>(yP, yQ, M, E, F, AL, scr, nullptr, nullptr, d, g, s_tab, sh, false);
            // A = F / E on interior nodes; weights h tan^2 sqrt(A); projections per mode (rank 0)
            const EigTab t = a.eig[d.geo];
            const double h = 1.0 / (12.0 * d.c12);
            const int lane = tid & 31, warp = tid >> 5;
            for (int j = warp; j < (rank == 0 ? a.J : 0); j += kANW) {
                double sp = 0.0, sf = 0.0;
                for (int i = 1 + lane; i < N - 1; i += 32) {
                    const double A = fma(-M[i], __ldg(g.K + i), 1.0);
                    const double w = h * __ldg(g.T + i) * sqrt(A);
                    sp = fma(w * yQ[i], __ldg(t.e + (size_t)j * N + i), sp);
                    sf = fma(w * yP[i], __ldg(t.de + (size_t)j * N + i), sf);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sp += __shfl_xor_sync(0xffffffffu, sp, o);
                    sf += __shfl_xor_sync(0xffffffffu, sf, o);
                }
                if (lane == 0) {
                    const double om = 3.0 + 2.0 * j, Eb = a.Ebar[(size_t)b * a.J + j];
                    scr.vP[j] = 2.0 * sp * Eb;              // Pi_j bar
                    scr.vQ[j] = 2.0 * sf * Eb / (om * om);  // Phi_j bar
                }
            }
            csync<CL>();
            if (act) {
#pragma unroll
                for (int k = 0; k < AP; ++k) {
                    const int i = i0 + k;
                    double cP = 0.0, cQ = 0.0, Ab = 0.0, dlb = 0.0;
                    if (i >= 1 && i < N - 1) {
                        double se = 0.0, sd = 0.0;
                        for (int j = 0; j < a.J; ++j) {
                            se = fma(scr.vP[j], __ldg(t.e + (size_t)j * N + i), se);
                            sd = fma(scr.vQ[j], __ldg(t.de + (size_t)j * N + i), sd);
                        }
                        const double A = fma(-M[i], __ldg(g.K + i), 1.0);
                        const double sa = sqrt(A), ht = h * __ldg(g.T + i);
                        cQ = ht * sa * se;
                        cP = ht * sa * sd;
                        Ab = ht * (yQ[i] * se + yP[i] * sd) / (2.0 * sa);
                    }
                    scr.ybP[i] = cP;
                    scr.ybQ[i] = cQ;
                    scr.mb[i] = -Ab * __ldg(g.K + i);
                    scr.dlb[i] = dlb;
                }
                if (own.last) { scr.mb[N - 1] = 0.0; scr.dlb[N - 1] = 0.0; }
            }
            csync<CL>();
            constraint_backward<CL, AP>(yP, yQ, M, AL, scr, scr.ybP, scr.ybQ, d, ag, sh);
            if (act) {
#pragma unroll
                for (int k = 0; k < AP; ++k) {
                    lamP[i0 + k] += scr.ybP[i0 + k];
                    lamQ[i0 + k] += scr.ybQ[i0 + k];
                }
            }
            csync<CL>();
            continue;
        }

        // ================= segment: phase F (recompute and store every stage) =================
        if (!SWEEP && (a.mode == kAdjSegment || a.mode == kAdjSegF)) {
        const double *ckP = a.ckP + d.off, *ckQ = a.ckQ + d.off;
        if (act) {
#pragma unroll
            for (int k = 0; k < AP; ++k) { scr.uP[i0 + k] = ckP[i0 + k]; scr.uQ[i0 + k] = ckQ[i0 + k]; }
        }
        csync<CL>();
        for (int n = 0; n < a.nsteps; ++n) {
            for (int s = 0; s < 4; ++s) {
                double *yP = slot(n, s, 0), *yQ = slot(n, s, 1);
                if (s == 0 && act) {
#pragma unroll
                    for (int k = 0; k < AP; ++k) { yP[i0 + k] = scr.uP[i0 + k]; yQ[i0 + k] = scr.uQ[i0 + k]; }
                }
                if (act && own.last) { yP[N - 1] = 0.0; yQ[N - 1] = 0.0; }
                csync<CL>();
                double *kP = scr.vP, *kQ = scr.vQ;   // stage derivative (phase F use of the slots)
                stage_forward<CL, AP>(yP, yQ, slot(n, s, 2), slot(n, s, 3), slot(n, s, 4), slot(n, s, 5), scr, kP, kQ,
                              d, g, s_tab, sh, true);
                if (act) {
#pragma unroll
                    for (int k = 0; k < AP; ++k) {
                        const int i = i0 + k;
                        const double up = scr.uP[i], uq = scr.uQ[i];
                        const double ap = (s == 0) ? fma(wst[0] * d.dt, kP[i], up) : fma(wst[s] * d.dt, kP[i], scr.aP[i]);
                        const double aq = (s == 0) ? fma(wst[0] * d.dt, kQ[i], uq) : fma(wst[s] * d.dt, kQ[i], scr.aQ[i]);
                        scr.aP[i] = ap;
                        scr.aQ[i] = aq;
                        if (s < 3) {
                            slot(n, s + 1, 0)[i] = fma(cst[s + 1] * d.dt, kP[i], up);
                            slot(n, s + 1, 1)[i] = fma(cst[s + 1] * d.dt, kQ[i], uq);
                        }
                    }
                }
                // no barrier: until the next stage's first barrier every thread touches only
                // its own nodes (the update reads the stage derivative of its own nodes)
            }
            if (act) {
#pragma unroll
                for (int k = 0; k < AP; ++k) { scr.uP[i0 + k] = scr.aP[i0 + k]; scr.uQ[i0 + k] = scr.aQ[i0 + k]; }
            }
        }
        if (a.outP && act) {   // the segment's last slice (the next segment's start)
            double *oP = a.outP + d.off, *oQ = a.outQ + d.off;
#pragma unroll
            for (int k = 0; k < AP; ++k) { oP[i0 + k] = scr.uP[i0 + k]; oQ[i0 + k] = scr.uQ[i0 + k]; }
            if (own.last) { oP[N - 1] = 0.0; oQ[N - 1] = 0.0; }
        }

        }   // phase F

        // ================= segment: phase B (steps backwards) =================
        if (SWEEP || a.mode == kAdjSegment || a.mode == kAdjSegB)
        for (int n = a.nsteps - 1; n >= 0; --n) {
            if (act) {
#pragma unroll
                for (int k = 0; k < AP; ++k) {
                    scr.lo[i0 + k] = lamP[i0 + k];
                    scr.lq[i0 + k] = lamQ[i0 + k];
                }
            }
            for (int s = 3; s >= 0; --s) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < AP; ++k) {
                        const int i = i0 + k;
                        // kbar, scaled by c12 (Phi) and cq (Pi): the factors of Phi-dot and Pi-dot
                        double kb = mul_f(s_kc[s][0], scr.lo[i]), kq = mul_f(s_kc[s][1], scr.lq[i]);
                        if (s < 3) {
                            kb = fma(s_kc[s][2], scr.ybP[i], kb);
                            kq = fma(s_kc[s][3], scr.ybQ[i], kq);
                        }
                        scr.vP[i] = (i == 0) ? 0.0 : kb;   // Phi-dot(0) is identically zero
                        scr.vQ[i] = kq;
                        scr.v2[i] = mul_f(agv(ag, kAgIT12k, i), kq);   // = iT12 kbar_Pi
                    }
                    if (own.last) { scr.vP[N - 1] = 0.0; scr.vQ[N - 1] = 0.0; scr.v2[N - 1] = 0.0; }
                }
                csync<CL>();
                stage_backward<CL, AP>(slot(n, s, 0), slot(n, s, 1), slot(n, s, 2), slot(n, s, 3), slot(n, s, 4),
                               slot(n, s, 5), scr, scr.ybP, scr.ybQ, d, ag, sh);
                if (act) {
#pragma unroll
                    for (int k = 0; k < AP; ++k) {
                        lamP[i0 + k] = add_f(lamP[i0 + k], scr.ybP[i0 + k]);
                        lamQ[i0 + k] = add_f(lamQ[i0 + k], scr.ybQ[i0 + k]);
                    }
                }
                // no barrier: the next stage first touches only this thread's nodes, then
                // synchronises before any neighbour read or before scr.pb, qb, r1, fb are rewritten
            }
        }
    }
}

}  // namespace adscl
