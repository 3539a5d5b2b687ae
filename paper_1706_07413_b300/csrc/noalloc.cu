// noalloc.cu -- adscl_evolve_noalloc: the batched evolution of adscl_evolve for callers that
// must not allocate device memory.
//
// Who needs it: a host program that hands all of the GPU's memory to its own pool at start-up
// and forbids allocations behind its back; code driven from a latency-critical loop, where the
// device-wide synchronisation of cudaMalloc/cudaFree cannot be tolerated; a plug-in called from
// inside another framework that owns every allocation.  Such callers pass their own device
// buffers for the fields and the results; everything else the evolution needs (geometry tables,
// RK4 accumulators, instance records, the work queue) lives in one fixed array below.
//
// The scratch array is a file-scope __device__ array, so every GPU that loads this library holds
// it (about 1.3 MB) until the process exits.  Host code may not use its name as an address: the
// device address is obtained once per device with cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "adscl.h"

// The kernels of evolve.cuh are instantiated here under a namespace of this file, so that this
// translation unit's copies do not collide with those of adscl.cu at link time.
namespace noalloc_impl {
#include "evolve.cuh"
}  // namespace noalloc_impl

using namespace noalloc_impl::adscl;

namespace {

constexpr int kNaP = 8;      // nodes per thread (same kernel shape as adscl_evolve)
constexpr int kNaNT = 512;   // threads per CTA
constexpr int kNaMaxN = kNaP * kNaNT + 1;                 // 4097
constexpr int kNaMaxB = ADSCL_NOALLOC_MAX_INSTANCES;      // 64
constexpr int kNaMaxPts = ADSCL_NOALLOC_MAX_POINTS;       // sum of N over the batch

// layout of the scratch array, in doubles
constexpr size_t kOffExp = 0;                                    // 256: 2^{j/256}
constexpr size_t kOffGeo = 256;                                  // 9 geometry tables
constexpr size_t kGeoLen = ((size_t)9 * ((kNaMaxN + 1) & ~1) + 31) / 32 * 32;
constexpr size_t kPtsLen = ((size_t)kNaMaxPts + 31) / 32 * 32;
constexpr size_t kOffAccP = kOffGeo + kGeoLen;                   // RK4 accumulator of Phi
constexpr size_t kOffAccQ = kOffAccP + kPtsLen;                  // RK4 accumulator of Pi
constexpr size_t kOffRec = kOffAccQ + kPtsLen;                   // instance records, queue
constexpr size_t kRecBytes = 16384;
constexpr size_t kScratchDoubles = kOffRec + kRecBytes / sizeof(double);

// byte offsets inside the record area
constexpr size_t kRecDesc = 0;
constexpr size_t kRecState = kRecDesc + sizeof(InstDesc) * kNaMaxB;
constexpr size_t kRecGeoTab = (kRecState + sizeof(InstState) * kNaMaxB + 255) / 256 * 256;
constexpr size_t kRecCtl = kRecGeoTab + 256;
constexpr size_t kRecRounds = kRecCtl + 256;
constexpr size_t kRecOrder = kRecRounds + sizeof(int32_t) * (kNaMaxB + 1);
constexpr size_t kRecEnd = kRecOrder + sizeof(int32_t) * kNaMaxB;
static_assert(kRecEnd <= kRecBytes, "record area too small");
static_assert((kOffRec * sizeof(double)) % 256 == 0, "record area alignment");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct DeviceSetup {
    bool ready = false;
    double *base = nullptr;  // device address of g_noalloc_scratch on this device
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Geometry factors of the grid x_i = i pi / (2 (N - 1)), same layout and definitions as the
// tables of adscl_create (ws, wt, K, T, iT12, wsm3, wtm, wsk, iT12k), computed here on the device.
__global__ void noalloc_geometry_kernel(double *t, int N, double sigma)
{
    const double h = 0.5 * 3.141592653589793 / (double)(N - 1);
    const int S = geo_stride(N);
    double *ws = t, *wt = ws + S, *K = wt + S, *T = K + S, *iT12 = T + S, *wsm3 = iT12 + S,
           *wtm = wsm3 + S, *wsk = wtm + S, *iT12k = wsk + S;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double x = i * h, s = sin(x), c = cos(x);
        ws[i] = h * s * c / 6.0;
        double Ti = 0.0;
        if (i < N - 1) {
            const double tn = tan(x);
            Ti = tn * tn;
        }
        T[i] = Ti;
        wt[i] = h * Ti / 6.0;
        K[i] = (i > 0 && i < N - 1) ? c * c * c / s : 0.0;
        iT12[i] = (i > 0 && i < N - 1) ? 1.0 / (12.0 * h * Ti) : 0.0;
        iT12k[i] = (i > 0 && i < N - 1) ? it12k_of(h, Ti, sigma) : 0.0;
        wsk[i] = kKappa * ws[i];
        if (i < N - 1) {
            const double xm = (i + 0.5) * h, sm = sin(xm), cm = cos(xm), tm = tan(xm);
            wsm3[i] = h * sm * cm / (2.0 * 256.0);
            wtm[i] = h * tm * tm / (6.0 * 256.0);
        } else {
            wsm3[i] = 0.0;
            wtm[i] = 0.0;
        }
    }
}

// The per-call records, written on the device from values passed by value (no host copy):
// instance b of the batch is the template `d` at offset b N; work item b runs instance b; the
// instance records start at zero (step 0, status RUNNING); one geometry table set.
__global__ void noalloc_records_kernel(InstDesc d, GeoTab g, int B, int N, InstDesc *desc,
                                       int32_t *order, GeoTab *geo, InstState *st)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) *geo = g;
    if (b >= B) return;
    InstDesc e = d;
    e.off = (int64_t)b * N;
    desc[b] = e;
    order[b] = b;
    InstState z;
    z.step = 0;
    z.t_c = 0.0;
    z.minA = 0.0;
    z.mass = 0.0;
    z.delta0 = 0.0;
    z.status = kRunning;
    z.pad = 0;
    st[b] = z;
}

__global__ void noalloc_exptab_kernel(double *tab)
{
    const int j = threadIdx.x;
    if (j < kExpTableSize) tab[j] = exp2((double)j / 256.0);
}

adscl_status setup_device(int device, double **base)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[device];
    if (!s.ready) {
        // the device must be current: the symbol address is per device
        if (cudaSetDevice(device) != cudaSuccess) return ADSCL_ECUDA;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return ADSCL_ECUDA;
        const size_t smem_max = (size_t)6 * field_stride<kNaP>(kNaMaxN) * sizeof(double);
        if (cudaFuncSetAttribute(evolve_kernel<kNaP, kNaNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_max) != cudaSuccess)
            return ADSCL_ECUDA;
        s.base = (double *)p;
        s.ready = true;
    }
    *base = s.base;
    return ADSCL_OK;
}

}  // namespace

extern "C" adscl_status adscl_evolve_noalloc(int32_t device, void *stream_, int32_t B, int32_t N,
                                             double *Phi, double *Pi, double t_end, double cfl,
                                             double ko_sigma, double collapse_threshold,
                                             double *t_reached, double *t_collapse, double *mass,
                                             int32_t *inst_status)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices)
        return ADSCL_EINVAL;
    if (!Phi || !Pi || !t_reached || !t_collapse || !mass || !inst_status) return ADSCL_EINVAL;
    if (N < 17 || (N - 1) % kNaP != 0 || !std::isfinite(t_end) || t_end < 0.0) return ADSCL_EINVAL;
    const double lam = cfl == 0.0 ? 0.5 : cfl;
    if (!(lam > 0.0 && lam <= 2.0) || !(ko_sigma >= 0.0 && ko_sigma < 10.0) ||
        !std::isfinite(collapse_threshold))
        return ADSCL_EINVAL;
    // fixed capacity of the scratch array
    if (B < 1 || B > kNaMaxB || N > kNaMaxN || (long long)B * N > kNaMaxPts) return ADSCL_ECAPACITY;
    // time step and the queue's round count, checked in floating point before any integer
    // conversion and before anything is queued (a t_end too long for the 32-bit ticket counter
    // is rejected here)
    constexpr int kChunk = 16;
    const double h = 0.5 * M_PI / (double)(N - 1);
    const double cad = 1.0;
    const double dt = cad / std::ceil(cad / (lam * h));
    const double n_end_d = std::ceil(t_end / dt - 1e-9);
    const double rounds_d = std::floor(n_end_d / kChunk) + 2.0;
    if (!(rounds_d * (double)B <= (double)0x7ffffff0)) return ADSCL_EINVAL;
    const int32_t rounds = (int32_t)rounds_d;

    double *base = nullptr;
    adscl_status st = setup_device(device, &base);
    if (st != ADSCL_OK) return st;
    if (cudaSetDevice(device) != cudaSuccess) return ADSCL_ECUDA;
    cudaStream_t stream = (cudaStream_t)stream_;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return ADSCL_ECUDA;

    char *rec = (char *)(base + kOffRec);
    InstDesc *d_desc = (InstDesc *)(rec + kRecDesc);
    InstState *d_st = (InstState *)(rec + kRecState);
    GeoTab *d_geo = (GeoTab *)(rec + kRecGeoTab);
    QueueCtl *d_ctl = (QueueCtl *)(rec + kRecCtl);
    int32_t *d_rounds = (int32_t *)(rec + kRecRounds);
    int32_t *d_order = (int32_t *)(rec + kRecOrder);
    double *geo = base + kOffGeo;

    // the instance template (every instance of the batch has the same grid and step)
    InstDesc desc{};
    desc.N = N;
    desc.geo = 0;
    desc.off = 0;
    set_desc_coeffs(desc, h, dt, ko_sigma);
    const size_t S = (size_t)geo_stride(N);
    GeoTab g;
    g.ws = geo;
    g.wt = geo + S;
    g.K = geo + 2 * S;
    g.T = geo + 3 * S;
    g.iT12 = geo + 4 * S;
    g.wsm3 = geo + 5 * S;
    g.wtm = geo + 6 * S;
    g.wsk = geo + 7 * S;
    g.iT12k = geo + 8 * S;

#define NA_CK(call) do { if ((call) != cudaSuccess) return ADSCL_ECUDA; } while (0)
    noalloc_records_kernel<<<1, kNaMaxB, 0, stream>>>(desc, g, B, N, d_desc, d_order, d_geo, d_st);
    NA_CK(cudaGetLastError());
    noalloc_exptab_kernel<<<1, kExpTableSize, 0, stream>>>(base + kOffExp);
    NA_CK(cudaGetLastError());
    noalloc_geometry_kernel<<<(N + 255) / 256, 256, 0, stream>>>(geo, N, ko_sigma);
    NA_CK(cudaGetLastError());

    EvolveArgs a{};
    a.desc = d_desc;
    a.st = d_st;
    a.geo = d_geo;
    a.exptab = base + kOffExp;
    a.Phi = Phi;
    a.Pi = Pi;
    a.aPhi = base + kOffAccP;
    a.aPi = base + kOffAccQ;
    a.order = d_order;
    a.nwork = B;
    a.chunk = kChunk;
    a.ctl = d_ctl;
    a.rounds = d_rounds;
    a.max_spin = (long long)1 << 24;
    a.t_end = t_end;
    a.theta = collapse_threshold;
    a.outA = nullptr;
    a.outDelta = nullptr;
    const int grid = B < sms ? B : sms;
    const int stride = field_stride<kNaP>(N);
    const size_t smem = (size_t)6 * stride * sizeof(double);

    // 1) initial slice: boundary values imposed, constraints solved (as adscl_set_initial)
    a.mode = kModeInit;
    a.max_rounds = 1;
    queue_init_kernel<<<1, 256, 0, stream>>>(d_ctl, d_rounds, B, grid);
    NA_CK(cudaGetLastError());
    evolve_kernel<kNaP, kNaNT><<<grid, kNaNT, smem, stream>>>(a, stride);
    NA_CK(cudaGetLastError());
    // 2) evolution to t_end or collapse (as adscl_evolve)
    a.mode = kModeEvolve;
    a.max_rounds = rounds;
    queue_init_kernel<<<1, 256, 0, stream>>>(d_ctl, d_rounds, B, grid);
    NA_CK(cudaGetLastError());
    evolve_kernel<kNaP, kNaNT><<<grid, kNaNT, smem, stream>>>(a, stride);
    NA_CK(cudaGetLastError());
    // 3) per-instance results straight into the caller's buffers
    gather_kernel<<<1, kNaMaxB, 0, stream>>>(d_desc, d_st, B, t_end, 1, d_ctl, d_order, t_reached,
                                             t_collapse, mass, inst_status);
    NA_CK(cudaGetLastError());
#undef NA_CK
    return ADSCL_OK;
}
