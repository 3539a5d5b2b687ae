// evolve_ea.cuh -- persistent FP64 kernel of the paper's production variant of the scheme
// (arXiv:1706.07413, Sec. II): A is evolved with Eq. (eq:adot) instead of being integrated from
// Eq. (eq:aprime) at every stage, and re-integrated from Eq. (eq:aprime) only every `reint`
// steps; delta is integrated from Eq. (eq:delta) at every stage; time stepping by the
// strong-stability-preserving Runge-Kutta methods of Shu and Osher of order 2 or 3,
//   y^{(s+1)} = a_s y_n + b_s (y^{(s)} + dt L(y^{(s)})),
//   order 2: (a, b) = (0, 1), (1/2, 1/2);  order 3: (0, 1), (3/4, 1/4), (1/3, 2/3).
//
// One CTA per instance (N <= P * NT + 1) or a cluster of CL = 2, 4, 8, 16 CTAs (N <= CL * P * NT + 1),
// with the layout, the ticket queue and the cluster protocol of evolve_kernel (halos, scan carries
// and slice diagnostics through distributed shared memory; control decisions by rank 0).
// Per stage:
//   1. cell data: the Simpson increments of delta (and, at a re-integration slice, the affine
//      maps of the mass function, as in evolve_kernel);
//   2. block suffix scan of delta (and the affine prefix scan at a re-integration slice);
//   3. F = A e^{-delta} with the stage's A, fluxes f = F Pi, u = tan^2 x F Phi, and
//      A-dot = -2 sin x cos x A F Phi Pi pointwise, which updates A at once (A has no spatial
//      derivative, so its stage value lives in an L2-resident global buffer, not in shared
//      memory);
//   4. Phi-dot, Pi-dot with dissipation as in evolve_kernel, Shu-Osher update.
// The state is (Phi, Pi, A) in global memory; the slice's diagnostics are min A, the mass
// M = int tan^2 x A rho dx by the composite Simpson rule on the nodes, and delta(0).
//
// FIXED = true: the fixed-metric case of the paper's Table II (A = 1 and delta = 0 held fixed,
// the linear wave equation on AdS4): no constraint phase, no scans, F = 1; the same RHS,
// dissipation and Shu-Osher update.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "evolve.cuh"

namespace adscl {

// per distinct grid size: the extra node factors of this scheme
struct EaGeo {            // two tables geo_stride(N) doubles apart (16-byte aligned)
    const double *K2;    // -2 sin x cos x                          (0 at both ends)
    const double *wsim;  // (h/3) w_i tan^2 x_i, w = Simpson weights (0 at both ends)
};

struct EaArgs {
    EvolveArgs e;        // e.aPhi: stage A buffer (packed like the fields); e.aPi unused
    const EaGeo *eg;
    double *A;           // packed evolved A (state)
    int32_t order;       // 2 or 3
    int32_t reint;       // re-integrate A from Eq. (eq:aprime) at slices n % reint == 0 (0: never)
};

template <int P, int NT, bool FIXED = false, int CL = 1>
__global__ void __launch_bounds__(NT, (NT >= 512) ? 1 : 512 / NT) evolve_ea_kernel(EaArgs ea, int stride)
{
    static_assert(P >= 4 && (P & (P - 1)) == 0, "P: power of two >= 4");
    static_assert(CL >= 1 && CL <= 16, "cluster of 1 to 16 CTAs");
    constexpr int NW = NT / 32;
    constexpr unsigned FULL = 0xffffffffu;
    const EvolveArgs &a = ea.e;
    extern __shared__ double smem[];
    double *bufA0 = smem, *bufA1 = smem + stride;                   // stage Phi, Pi
    double *bufB0 = smem + 2 * stride, *bufB1 = smem + 3 * stride;  // next stage Phi, Pi
    double *sF = smem + 4 * stride, *sU = smem + 5 * stride;        // alpha/beta, then f/u
    __shared__ double s_tab[kExpTableSize];
    __shared__ double wAl[NW], wBe[NW], wDe[NW], cM[NW], cMa[NW], cD[NW], wMs[NW];
    __shared__ long long wMin[NW], wMinP[CL * NW];
    __shared__ double wMsP[CL * NW];
    __shared__ double s_d0, s_cA[CL], s_cB[CL], s_cD[CL];
    __shared__ int s_cmd, s_q, s_r, s_leave, s_status;
    __shared__ long long s_step;
    __shared__ double s_tc, s_minA, s_massS, s_d0S;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int rank = 0;
    if constexpr (CL > 1) rank = cluster_rank();
    for (int i = tid; i < kExpTableSize; i += NT) s_tab[i] = a.exptab[i];
    csync<CL>();   // every CTA of the cluster has started before any remote shared-memory store

    for (;;) {
        // ------------------------------------------------------------ take a ticket
        if (tid == 0 && rank == 0) {
            int cmd = 0, q = 0, r = 0;
            for (;;) {
                if (ld_relaxed(&a.ctl->unfinished) == 0 || ld_relaxed(&a.ctl->error) != 0) break;
                const int t = atomicAdd(&a.ctl->ticket, 1);
                if (t >= a.nwork * a.max_rounds) break;
                r = t / a.nwork;
                q = t - r * a.nwork;
                int rd = ld_acquire(a.rounds + q);
                long long spin = 0;
                while (rd < r) {
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
        const int Nl = N - gb;             // local index of node N
        const GeoTab g = a.geo[d.geo];
        const EaGeo eg = ea.eg[d.geo];
        double *uPhi = a.Phi + d.off, *uPi = a.Pi + d.off, *uA = ea.A + d.off;
        double *sA = a.aPhi + d.off;   // stage A (entry k of node block t at k * TnAll + t)
        const bool skip = (a.mode == kModeEvolve) && (S.status != kRunning || S.step >= n_target);
        const int R = ea.order;

        long long step = S.step;
        double minA_prev = S.minA, minA = S.minA, mass = S.mass, d0 = S.delta0, t_c = S.t_c;
        int32_t status = S.status;

        if (!skip) {
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
                        uA[N - 1] = 1.0;
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
                for (int s = 0; s < R; ++s) {
                    // the initial slice always takes A from the constraint
                    const bool reint = !FIXED && (s == 0) && (a.mode == kModeInit ||
                                                              (ea.reint > 0 && step % ea.reint == 0));
                    const double wa = (s == 0) ? 0.0 : (R == 2 ? 0.5 : (s == 1 ? 0.75 : 1.0 / 3.0));
                    const double wb = (s == 0) ? 1.0 : (R == 2 ? 0.5 : (s == 1 ? 0.25 : 2.0 / 3.0));
                    // ================= delta (and, at a re-integration slice, m) =================
                    double De[P];
                    double aT = 1.0, bT = 0.0, SD = 0.0;
                    double aEx = 1.0, bEx = 0.0;
                    if constexpr (!FIXED) {
                    if (act) {
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        double pm1 = Sp[soff<P>(-1)], p0 = Sp[soff<P>(0)], p1 = Sp[soff<P>(1)];
                        double qm1 = Sq[soff<P>(-1)], q0 = Sq[soff<P>(0)], q1 = Sq[soff<P>(1)];
                        double gws[P + 1], gwm[P];   // wsk at nodes i0 .. i0+P, wsm3 at cells i0 ..
                        ldg_run<P>(g.wsk + i0, gws);
                        ldg_run<P>(g.wsm3 + i0, gwm);
                        gws[P] = __ldg(g.wsk + i0 + P);
                        const double rho0 = fma(p0, p0, mul_f(q0, q0));
                        double qn0 = mul_f(gws[0], rho0), rn0 = mul_f(__ldg(g.wt + i0), rho0);
                        // compiled once with the mass map (re-integration slices) and once without
                        auto cell_nodes = [&](auto with_map) {
                        constexpr bool REINT = decltype(with_map)::value;
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int c = i0 + k;
                            const double p2 = Sp[soff<P>(k + 2)], q2 = Sq[soff<P>(k + 2)];
                            const double rho1 = fma(p1, p1, mul_f(q1, q1));
                            const double qn1 = mul_f(gws[k + 1], rho1);   // kappa q1
                            const double p16 = fma(9.0, add_f(p0, p1), -add_f(pm1, p2));
                            const double q16 = fma(9.0, add_f(q0, q1), -add_f(qm1, q2));
                            const double rm = fma(p16, p16, mul_f(q16, q16));
                            const double qm3 = mul_f(gwm[k], rm);
                            const double s01 = add_f(qn0, qn1);
                            const double dek = fma(kKappa * (4.0 / 3.0), qm3, s01);   // units of ln2/256
                            // De[k] (k >= 1): sum of the increments of cells i0 .. i0+k-1
                            if (k > 0) De[k] = SD;
                            SD = (k == 0) ? dek : add_f(SD, dek);
                            if constexpr (REINT) {
                                // the affine map of the mass function over the cell (evolve_kernel)
                                const double rn1 = mul_f(__ldg(g.wt + c + 1), rho1);
                                const double tm = mul_f(__ldg(g.wtm + c), rm);
                                const double y2 = fma(-kInvKappa, qn0, 1.0 / 3.0);
                                const double y3 = fma(-qm3, y2, 1.0 / 3.0);
                                const double ca = fma(-6.0 * kInvKappa, qn1, 2.0);
                                const double e = fma(-qm3, ca, 2.0);
                                const double al = fma(y3, e, fma(-kInvKappa, s01, 1.0 / 3.0));
                                const double w2 = fma(-qm3, rn0, tm);
                                const double be = fma(e, w2, fma(ca, tm, add_f(rn0, rn1)));
                                sF[tb + soff<P>(k)] = al;
                                sU[tb + soff<P>(k)] = be;
                                if (k == 0) {
                                    aT = al;
                                    bT = be;
                                } else {
                                    bT = fma(al, bT, be);
                                    aT = mul_f(aT, al);
                                }
                                rn0 = rn1;
                            }
                            pm1 = p0; p0 = p1; p1 = p2;
                            qm1 = q0; q0 = q1; q1 = q2;
                            qn0 = qn1;
                        }
                        };
                        if (reint) cell_nodes(std::true_type{});
                        else cell_nodes(std::false_type{});
                    }
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const double dn = __shfl_down_sync(FULL, SD, o);
                        if (lane + o < 32) SD = add_f(SD, dn);
                    }
                    if (reint) {
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const double ap = __shfl_up_sync(FULL, aT, o);
                            const double bp = __shfl_up_sync(FULL, bT, o);
                            if (lane >= o) {
                                bT = fma(aT, bp, bT);
                                aT = mul_f(aT, ap);
                            }
                        }
                    }
                    aEx = __shfl_up_sync(FULL, aT, 1);
                    bEx = __shfl_up_sync(FULL, bT, 1);
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
                                A_ = mul_f(A_, ap);
                            }
                            if (lane + o < NW) D_ = add_f(D_, dn);
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
                            // block totals to the other ranks: the m map to higher ranks (only read
                            // on re-integration slices), the delta sum to lower ranks
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
                    }   // !FIXED

                    // ============ fluxes, A-dot and the A update; diagnostics of the slice ============
                    long long kmin = 0x7FFFFFFFFFFFFFFFLL;
                    double msum = 0.0;
                    if (act) {
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        double m = 0.0;
                        if constexpr (FIXED) {
#pragma unroll
                            for (int k = 0; k < P; ++k) De[k] = 0.0;
                        } else {
                            double cm = cM[wid], dr = 0.0;
                            if constexpr (CL > 1) {
                                // m at this rank's first node: the maps of the ranks before it
                                double mr = 0.0;
                                for (int j = 0; j < rank; ++j) mr = (j == 0) ? s_cB[0] : fma(s_cA[j], mr, s_cB[j]);
                                if (rank > 0) cm = fma(cMa[wid], mr, cm);
                                // delta carried in from the ranks to the right
                                for (int j = CL - 1; j > rank; --j) dr = (j == CL - 1) ? s_cD[j] : dr + s_cD[j];
                            }
                            m = fma(aEx, cm, bEx);
                            // delta at node i0 from the inclusive suffix sum SD, then at node i0+k
                            // by subtracting the increments of the cells i0 .. i0+k-1
                            const double dtop = add_f(add_f(SD, cD[wid]), dr);
                            De[0] = dtop;
#pragma unroll
                            for (int k = 1; k < P; ++k) De[k] = add_f(dtop, -De[k]);
                        }
                        double g1 = 0.0, g2 = 0.0, um1 = 0.0, um2 = 0.0, fm1 = 0.0, fm2 = 0.0;
                        double f0 = 0.0, f1 = 0.0, u0 = 0.0, u1 = 0.0;
                        double gT[P], gK2[P];
                        ldg_run<P>(g.T + i0, gT);
                        if constexpr (!FIXED) ldg_run<P>(eg.K2 + i0, gK2);
                        // the node loop, compiled once for the first stage of a step and once for the later
                        // stages, so that no stage issues the other's FP64 work with its lanes predicated off
                        auto flux_nodes = [&](auto first_stage) {
                        constexpr bool FIRST = decltype(first_stage)::value;
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int i = i0 + k;
                            const double ph = Sp[soff<P>(k)], pi = Sq[soff<P>(k)];
                            double Ai;
                            if (FIXED) {
                                Ai = 1.0;
                            } else if (FIRST && reint) {   // re-integration slices are first stages
                                const double al = sF[tb + soff<P>(k)], be = sU[tb + soff<P>(k)];
                                Ai = fma(-m, __ldg(g.K + i), 1.0);
                                uA[i] = Ai;   // the slice's A is the constraint solution
                                if (k < P - 1) m = fma(al, m, be);
                            } else {
                                Ai = FIRST ? __ldcg(uA + i) : __ldcg(sA + k * TnAll + bs + tid);
                            }
                            const double Fi = FIXED ? 1.0 : a_exp_neg_scaled(Ai, De[k], s_tab);
                            const double gi = FIXED ? ph : mul_f(Fi, ph);
                            const double fi = FIXED ? pi : mul_f(Fi, pi);
                            const double ui = mul_f(gT[k], gi);
                            if constexpr (!FIXED) {
                                // A-dot = -2 sin x cos x A (A e^{-delta} Phi) Pi, and the stage update
                                const double dA = mul_f(mul_f(mul_f(gK2[k], Ai), gi), pi);
                                const double An = FIRST ? fma(dt, dA, Ai)
                                                           : fma(wb, fma(dt, dA, Ai), mul_f(wa, __ldcg(uA + i)));
                                if (s < R - 1) sA[k * TnAll + bs + tid] = An;
                                else uA[i] = An;
                            }
                            if constexpr (FIRST) {
                                kmin = min_ll(kmin, order_key(Ai));
                                msum = FIXED ? fma(__ldg(eg.wsim + i), fma(ph, ph, mul_f(pi, pi)), msum)
                                             : fma(mul_f(__ldg(eg.wsim + i), Ai), fma(ph, ph, mul_f(pi, pi)), msum);
                            }
                            sF[tb + soff<P>(k)] = fi;
                            sU[tb + soff<P>(k)] = ui;
                            if (k == 0) { f0 = fi; u0 = ui; }
                            if (k == 1) { g1 = gi; f1 = fi; u1 = ui; }
                            if (k == 2) g2 = gi;
                            if (tfirst && (k == 1 || k == 2)) {
                                sF[spos<P>(-k)] = fi;
                                sU[spos<P>(-k)] = neg_bits(ui);
                            }
                            if (k == P - 1) { fm1 = fi; um1 = ui; }
                            if (k == P - 2) { fm2 = fi; um2 = ui; }
                            if (a.outA) {
                                a.outA[d.off + i] = Ai;
                                a.outDelta[d.off + i] = De[k];   // in units of ln2/256 (no FP64 work here)
                            }
                        }
                        };
                        if (s == 0) flux_nodes(std::true_type{});
                        else flux_nodes(std::false_type{});
                        // the grid's two ends, in a branch that only their warps take
                        if (__any_sync(__activemask(), tfirst || last)) {
                        if (tfirst) {
                            const double d0n = De[0] * kInvKappa;   // delta(0)
                            s_d0 = d0n;
                            sF[spos<P>(-3)] = fma(16.0, g1, -2.0 * g2);
                            if constexpr (CL > 1) st_others<CL>(&s_d0, d0n, 0);
                        }
                        if (last) {
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
                    if (s == 0) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            kmin = min_ll(kmin, __shfl_xor_sync(FULL, kmin, o));
                            msum += __shfl_xor_sync(FULL, msum, o);
                        }
                        if (lane == 0) {
                            wMin[wid] = kmin;
                            wMs[wid] = msum;
                            if constexpr (CL > 1) {
                                st_others<CL>(wMinP + rank * NW + wid, kmin, rank);
                                st_others<CL>(wMsP + rank * NW + wid, msum, rank);
                            }
                        }
                    }
                    csync<CL>();

                    if (s == 0) {
                        long long km = wMin[0];
                        double ms = 0.0;
                        // the same summation order on every rank: ranks ascending, warps ascending
#pragma unroll 1
                        for (int j = 0; j < CL; ++j) {
                            const long long *wk = (j == rank) ? wMin : wMinP + j * NW;
                            const double *wm = (j == rank) ? wMs : wMsP + j * NW;
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                km = min_ll(km, wk[w]);
                                ms = (j == 0 && w == 0) ? wm[0] : ms + wm[w];
                            }
                        }
                        minA = order_key_inv(km);
                        mass = ms;
                        d0 = s_d0;
                        const bool nonfin = !(is_finite_bits(mass) && is_finite_bits(d0) && is_finite_bits(minA));
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

                    // ================= Phi-dot, Pi-dot and the Shu-Osher update =================
                    if (act) {
                        const double wbdc = wb * d.dtc, wbd = wb * d.dtq;
                        const double *Sp = S0 + tb, *Sq = S1 + tb;
                        const double *f = sF + tb, *u = sU + tb;
                        double *Dp = D0 + tb, *Dq = D1 + tb;
                        double gI[P];
                        ldg_run<P>(g.iT12k + i0, gI);
                        // compiled per stage kind as the flux loop
                        auto update_nodes = [&](auto first_stage) {
                        constexpr bool FIRST = decltype(first_stage)::value;
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
                            double Xp = fma(d.rko, kp, Df);   // Phi-dot / c12
                            const double kqs = d.ko ? kq : 0.0;
                            double dQ = fma(gI[k], Du, kqs);   // Pi-dot / cq
                            if (k == 0 && tfirst) {
                                Xp = 0.0;
                                dQ = fma(d.c3q, sF[spos<P>(-3)], kqs);
                            }
                            double np, nq;
                            if constexpr (FIRST) {
                                np = fma(d.dtc, Xp, Sp[soff<P>(k)]);
                                nq = fma(d.dtq, dQ, Sq[soff<P>(k)]);
                            } else {
                                np = fma(wbdc, Xp, fma(wb, Sp[soff<P>(k)], mul_f(wa, __ldcg(uPhi + i))));
                                nq = fma(wbd, dQ, fma(wb, Sq[soff<P>(k)], mul_f(wa, __ldcg(uPi + i))));
                            }
                            if (k == 0 && tfirst) np = 0.0;
                            if (s == R - 1) {
                                uPhi[i] = np;
                                uPi[i] = nq;
                            }
                            Dp[soff<P>(k)] = np;
                            Dq[soff<P>(k)] = nq;
                            if (tfirst && k >= 1 && k <= 3) {
                                D0[spos<P>(-k)] = neg_bits(np);
                                D1[spos<P>(-k)] = nq;
                            }
                            if (last && k >= P - 3) {
                                D0[spos<P>(Nl - 1 + (P - k))] = np;
                                D1[spos<P>(Nl - 1 + (P - k))] = neg_bits(nq);
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
                        if (s == 0) update_nodes(std::true_type{});
                        else update_nodes(std::false_type{});
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
        csync<CL>();   // all global writes of this chunk are issued, by every CTA of the cluster
        if (tid == 0 && rank == 0) {
            if (!skip) {
                InstState *spw = a.st + b;
                spw->step = step;
                spw->t_c = t_c;
                spw->minA = minA;
                spw->mass = mass;
                spw->delta0 = d0;
                spw->status = status;
            }
            __threadfence();
            const bool fin = (a.mode != kModeEvolve) || status != kRunning || step >= n_end;
            if (fin) {
                atomicExch(a.rounds + q, kFinished);
                atomicSub(&a.ctl->unfinished, 1);
            } else {
                atomicExch(a.rounds + q, rnd + 1);
            }
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

}  // namespace adscl
