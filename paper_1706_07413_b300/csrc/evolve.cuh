// evolve.cuh -- persistent FP64 method-of-lines kernel for the AdS4 Einstein-Klein-Gordon
// system of arXiv:1706.07413, Sec. II (Eqs. (eq:phi), (eq:pi), (eq:aprime), (eq:delta)).
//
// One CTA evolves one instance at a time with the whole stage slice resident in shared
// memory; CTAs pull instances from an atomic work queue (persistent grid, one CTA per SM).
// Thread t owns the P contiguous grid nodes t*P .. t*P+P-1 and the cells to their right;
// node N-1 (x = pi/2, where Phi = Pi = 0) is owned by nobody and written as a constant.
//
// Per RK stage:
//   1. cell data: rho at nodes and (4-point interpolated) midpoints, the Simpson increment
//      Delta_c of Eq. (eq:delta) and the RK4-in-x affine map m -> alpha_c m + beta_c of the
//      mass-function form of Eq. (eq:aprime);
//   2. a block scan: delta as a suffix sum of Delta, m as a prefix composition of affine maps
//      (per-thread serial, then warp shuffles, then one warp over the warp totals);
//   3. A = 1 - m cos^3 x / sin x, F = A e^{-delta}, fluxes f = F Pi and u = tan^2 x F Phi;
//   4. RHS: Phi-dot = D f, Pi-dot = D u / tan^2 x (Eq. (eq:pi) in its conservative form),
//      Kreiss-Oliger dissipation, classic RK4 accumulation.
// The FP64 pipe is the bound on this chip, so every term is arranged to minimise FP64
// instructions; comparisons and finiteness tests run on the integer pipe.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace adscl {

constexpr int kG = 4;  // ghost padding on each side of the shared-memory field arrays

// per distinct grid size: geometry factors at nodes (length N) and cell midpoints (N-1)
struct GeoTab {
    const double *ws;    // h sin x cos x / 6
    const double *wt;    // h tan^2 x / 6            (0 at x = pi/2)
    const double *K;     // cos^3 x / sin x          (0 at both ends)
    const double *T;     // tan^2 x                  (0 at x = pi/2)
    const double *iT12;  // 1 / (12 h tan^2 x)       (0 at both ends)
    const double *wsm;   // h sin x cos x / (6*256) at x_{c+1/2}
    const double *wtm;   // h tan^2 x / (6*256)     at x_{c+1/2}
};

struct InstDesc {
    int32_t N;
    int32_t geo;
    int64_t off;  // offset of this instance in the packed field arrays
    double dt, dt2, dt3, dt6;
    double c12;   // 1 / (12 h)
    double c3;    // 3 / (12 h)
    double cko;   // sigma / (64 h)
};

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

struct EvolveArgs {
    const InstDesc *desc;
    InstState *st;
    const GeoTab *geo;
    double *Phi, *Pi;     // packed current slices (updated in place)
    double *aPhi, *aPi;   // packed RK4 accumulators (workspace)
    const int32_t *order; // work item -> instance
    int32_t nwork;
    int32_t *queue;       // work counter, zero before the launch
    double t_end;
    double theta;
    double *outA, *outDelta;  // kModeSolve only: packed A, delta of the slice (may be null)
    int32_t mode;
};

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

template <int P, int NT>
__global__ void __launch_bounds__(NT, 1) evolve_kernel(EvolveArgs a, int stride)
{
    static_assert(P >= 4, "ghost fill needs >= 4 nodes per thread");
    constexpr int NW = NT / 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ double smem[];
    double *sPhi = smem;
    double *sPi = sPhi + stride;
    double *sF = sPi + stride;
    double *sU = sF + stride;
    __shared__ double wAl[NW], wBe[NW], wDe[NW], cM[NW], cD[NW];
    __shared__ long long wMin[NW];
    __shared__ double s_mass, s_d0;
    __shared__ int s_item;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.nwork) break;
        const int b = a.order[item];
        const InstDesc d = a.desc[b];
        InstState S = a.st[b];
        const double dt = d.dt;
        long long n_end = 0;
        if (a.mode == kModeEvolve) {
            if (S.status != kRunning) continue;
            n_end = (long long)ceil(a.t_end / dt - 1e-9);
            if (S.step >= n_end) continue;
        }
        const int N = d.N;
        const int Tn = (N - 1) / P;
        const bool act = tid < Tn;
        const bool last = tid == Tn - 1;
        const int i0 = tid * P;
        const GeoTab g = a.geo[d.geo];
        double *uPhi = a.Phi + d.off, *uPi = a.Pi + d.off;
        double *cPhi = a.aPhi + d.off, *cPi = a.aPi + d.off;

        // ---- load the current slice into the stage arrays (boundary values imposed) ----
        {
            double p[P], q[P];
            if (act) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    p[k] = uPhi[i0 + k];
                    q[k] = uPi[i0 + k];
                }
                if (tid == 0) p[0] = 0.0;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    sPhi[kG + i0 + k] = p[k];
                    sPi[kG + i0 + k] = q[k];
                }
                if (tid == 0) {
#pragma unroll
                    for (int j = 1; j <= 3; ++j) {
                        sPhi[kG - j] = -p[j];
                        sPi[kG - j] = q[j];
                    }
                    if (a.mode == kModeInit) uPhi[0] = 0.0;
                }
                if (last) {
                    sPhi[kG + N - 1] = 0.0;
                    sPi[kG + N - 1] = 0.0;
#pragma unroll
                    for (int j = 1; j <= 3; ++j) {
                        sPhi[kG + N - 1 + j] = p[P - j];
                        sPi[kG + N - 1 + j] = -q[P - j];
                    }
                    if (a.mode == kModeInit) {
                        uPhi[N - 1] = 0.0;
                        uPi[N - 1] = 0.0;
                    }
                }
            }
        }
        __syncthreads();

        long long step = S.step;
        double minA_prev = S.minA, minA = S.minA, mass = S.mass, d0 = S.delta0, t_c = S.t_c;
        int32_t status = S.status;
        bool first = true;

        for (;;) {
#pragma unroll 1
            for (int s = 0; s < 4; ++s) {
                // ================= constraint solve on the stage slice =================
                double al[P], be[P], De[P];
                double aT = 1.0, bT = 0.0, SD = 0.0;
                if (act) {
                    double ph[P + 3], pq[P + 3];  // nodes i0-1 .. i0+P+1
#pragma unroll
                    for (int k = 0; k < P + 3; ++k) {
                        ph[k] = sPhi[kG + i0 - 1 + k];
                        pq[k] = sPi[kG + i0 - 1 + k];
                    }
                    double qn[P + 1], rn[P + 1];  // per node: h s rho / 6, h tan^2 rho / 6
#pragma unroll
                    for (int k = 0; k <= P; ++k) {
                        const double rho = fma(ph[k + 1], ph[k + 1], pq[k + 1] * pq[k + 1]);
                        qn[k] = __ldg(g.ws + i0 + k) * rho;
                        rn[k] = __ldg(g.wt + i0 + k) * rho;
                    }
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const int c = i0 + k;
                        // 16 * (midpoint value) by the 4-point Lagrange formula
                        const double p16 = fma(9.0, ph[k + 1] + ph[k + 2], -(ph[k] + ph[k + 3]));
                        const double q16 = fma(9.0, pq[k + 1] + pq[k + 2], -(pq[k] + pq[k + 3]));
                        const double rm = fma(p16, p16, q16 * q16);  // 256 rho_{c+1/2}
                        const double qm = __ldg(g.wsm + c) * rm;     // h s rho / 6 at the midpoint
                        const double tm = __ldg(g.wtm + c) * rm;     // h tan^2 rho / 6 at the midpoint
                        // Simpson increment of delta over the cell
                        De[k] = fma(4.0, qm, qn[k] + qn[k + 1]);
                        // RK4 in x of m' = a - b m over the cell, as the affine map
                        // m -> alpha m + beta (alpha: y' = -b y, y = 1; beta: y' = a - b y, y = 0)
                        const double qm3 = 3.0 * qm;
                        const double y2 = fma(-3.0, qn[k], 1.0);
                        const double y3 = fma(-qm3, y2, 1.0);
                        const double y4 = fma(-2.0 * qm3, y3, 1.0);
                        al[k] = fma(-2.0 * qm, y2 + y3, fma(-qn[k + 1], y4, 1.0 - qn[k]));
                        const double w2 = fma(-qm3, rn[k], tm);
                        const double w3 = fma(-qm, 3.0 * w2, tm);
                        const double w4 = fma(-qn[k + 1], 6.0 * w3, rn[k + 1]);
                        be[k] = fma(2.0, w2 + w3, rn[k]) + w4;
                    }
                    aT = al[0];
                    bT = be[0];
                    SD = De[0];
#pragma unroll
                    for (int k = 1; k < P; ++k) {
                        bT = fma(al[k], bT, be[k]);
                        aT = aT * al[k];
                        SD = SD + De[k];
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
                        aT = aT * ap;
                    }
                    if (lane + o < 32) SD = SD + dn;
                }
                double aEx = __shfl_up_sync(FULL, aT, 1);
                double bEx = __shfl_up_sync(FULL, bT, 1);
                double dEx = __shfl_down_sync(FULL, SD, 1);
                if (lane == 0) { aEx = 1.0; bEx = 0.0; }
                if (lane == 31) dEx = 0.0;
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
                }
                __syncthreads();

                long long kmin = 0x7FFFFFFFFFFFFFFFLL;
                if (act) {
                    double m = fma(aEx, cM[wid], bEx);   // m at node i0
                    double dl[P];                        // delta at nodes i0 .. i0+P-1
                    double dc = dEx + cD[wid];           // delta at node i0+P
#pragma unroll
                    for (int k = P - 1; k >= 0; --k) {
                        dc = dc + De[k];
                        dl[k] = dc;
                    }
                    double fv[P], uv[P];
                    double g1 = 0.0, g2 = 0.0;
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const int i = i0 + k;
                        const double Ai = fma(-m, __ldg(g.K + i), 1.0);
                        kmin = min_ll(kmin, order_key(Ai));
                        const double Fi = Ai * exp(-dl[k]);
                        const double phi = sPhi[kG + i], pii = sPi[kG + i];
                        const double gi = Fi * phi;
                        fv[k] = Fi * pii;
                        uv[k] = __ldg(g.T + i) * gi;
                        if (k == 1) g1 = gi;
                        if (k == 2) g2 = gi;
                        sF[kG + i] = fv[k];
                        sU[kG + i] = uv[k];
                        if (a.outA) {
                            a.outA[d.off + i] = Ai;
                            a.outDelta[d.off + i] = dl[k];
                        }
                        if (k < P - 1) m = fma(al[k], m, be[k]);
                    }
                    if (tid == 0) {
                        s_d0 = dl[0];
                        sF[kG - 1] = fv[1];
                        sF[kG - 2] = fv[2];
                        sU[kG - 1] = -uv[1];
                        sU[kG - 2] = -uv[2];
                        // Pi-dot at x = 0 needs (F Phi)'(0) = (16 g_1 - 2 g_2) / (12 h)
                        sF[kG - 3] = fma(16.0, g1, -2.0 * g2);
                    }
                    if (last) {
                        s_mass = fma(al[P - 1], m, be[P - 1]);
                        sF[kG + N - 1] = 0.0;
                        sF[kG + N] = -fv[P - 1];
                        sF[kG + N + 1] = -fv[P - 2];
                        sU[kG + N - 1] = (4.0 * uv[P - 1] - uv[P - 2]) * (1.0 / 3.0);
                        sU[kG + N] = uv[P - 1];
                        sU[kG + N + 1] = uv[P - 2];
                        if (a.outA) {
                            a.outA[d.off + N - 1] = 1.0;
                            a.outDelta[d.off + N - 1] = 0.0;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) kmin = min_ll(kmin, __shfl_xor_sync(FULL, kmin, o));
                if (lane == 0) wMin[wid] = kmin;
                __syncthreads();

                if (s == 0) {
                    // ---------- end-of-step diagnostics on the slice t = step * dt ----------
                    long long km = wMin[0];
#pragma unroll
                    for (int w = 1; w < NW; ++w) km = min_ll(km, wMin[w]);
                    minA = order_key_inv(km);
                    mass = s_mass;
                    d0 = s_d0;
                    const bool nonfin = !(is_finite_bits(mass) && is_finite_bits(d0));
                    bool stop = false;
                    if (a.mode != kModeEvolve) {
                        if (a.mode == kModeInit) {
                            status = nonfin ? kNonfinite : (minA < a.theta ? kCollapsed : kRunning);
                            t_c = (status == kCollapsed) ? 0.0 : __longlong_as_double(0x7FF0000000000000LL);
                        }
                        stop = true;
                    } else if (!first) {
                        if (nonfin) {
                            status = kNonfinite;
                            stop = true;
                        } else if (minA < a.theta) {
                            // min A crossed theta between t_{n-1} and t_n: linear interpolation
                            t_c = (double)(step - 1) * dt + dt * (minA_prev - a.theta) / (minA_prev - minA);
                            status = kCollapsed;
                            stop = true;
                        }
                    }
                    if (!stop && step >= n_end) stop = true;
                    if (stop) goto finish;
                    minA_prev = minA;
                    first = false;
                }

                // ================= right-hand side and RK4 update =================
                {
                    double nP[P], nQ[P];
                    if (act) {
                        const double wacc = (s == 0 || s == 3) ? d.dt6 : d.dt3;
                        const double wst = (s == 2) ? dt : d.dt2;
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int i = i0 + k;
                            const double *f = sF + kG + i, *u = sU + kG + i;
                            const double *p = sPhi + kG + i, *q = sPi + kG + i;
                            const double Df = (f[-2] - f[2]) + 8.0 * (f[1] - f[-1]);
                            const double Du = (u[-2] - u[2]) + 8.0 * (u[1] - u[-1]);
                            double kp = fma(-20.0, p[0], fma(15.0, p[-1] + p[1], fma(-6.0, p[-2] + p[2], p[-3] + p[3])));
                            double kq = fma(-20.0, q[0], fma(15.0, q[-1] + q[1], fma(-6.0, q[-2] + q[2], q[-3] + q[3])));
                            double dP = fma(d.c12, Df, d.cko * kp);
                            double dQ = fma(__ldg(g.iT12 + i), Du, d.cko * kq);
                            if (k == 0 && tid == 0) {
                                dP = 0.0;                                // Phi(0) = 0
                                dQ = fma(d.c3, sF[kG - 3], d.cko * kq);  // Pi-dot(0) = 3 (F Phi)'(0)
                            }
                            const double up = uPhi[i], uq = uPi[i];
                            double ap_, aq_;
                            if (s == 0) {
                                ap_ = fma(wacc, dP, up);
                                aq_ = fma(wacc, dQ, uq);
                            } else {
                                ap_ = fma(wacc, dP, cPhi[i]);
                                aq_ = fma(wacc, dQ, cPi[i]);
                            }
                            if (s < 3) {
                                cPhi[i] = ap_;
                                cPi[i] = aq_;
                                nP[k] = fma(wst, dP, up);
                                nQ[k] = fma(wst, dQ, uq);
                            } else {
                                nP[k] = ap_;
                                nQ[k] = aq_;
                                uPhi[i] = ap_;
                                uPi[i] = aq_;
                            }
                        }
                    }
                    __syncthreads();
                    if (act) {
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            sPhi[kG + i0 + k] = nP[k];
                            sPi[kG + i0 + k] = nQ[k];
                        }
                        if (tid == 0) {
#pragma unroll
                            for (int j = 1; j <= 3; ++j) {
                                sPhi[kG - j] = -nP[j];
                                sPi[kG - j] = nQ[j];
                            }
                        }
                        if (last) {
#pragma unroll
                            for (int j = 1; j <= 3; ++j) {
                                sPhi[kG + N - 1 + j] = nP[P - j];
                                sPi[kG + N - 1 + j] = -nQ[P - j];
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            ++step;
        }
    finish:
        if (tid == 0) {
            S.step = step;
            S.t_c = t_c;
            S.minA = minA;
            S.mass = mass;
            S.delta0 = d0;
            S.status = status;
            a.st[b] = S;
        }
        __syncthreads();
    }
}

// per-instance results of an evolve call: t_reached, t_collapse, mass, status
__global__ void gather_kernel(const InstDesc *desc, const InstState *st, int B, double t_end,
                              int evolve_call, double *t_reached, double *t_c, double *mass,
                              int32_t *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const InstState S = st[b];
    t_reached[b] = (double)S.step * desc[b].dt;
    t_c[b] = S.t_c;
    mass[b] = S.mass;
    int32_t s = S.status;
    if (evolve_call && s == kRunning) {
        const long long n_end = (long long)ceil(t_end / desc[b].dt - 1e-9);
        if (S.step >= n_end) s = kDone;
    }
    status[b] = s;
}

}  // namespace adscl
