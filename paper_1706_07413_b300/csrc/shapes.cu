// shapes.cu -- instantiations of the evolution kernel for every shape in kShapes, their
// occupancy queries and launches (kept in their own translation unit so that they compile in
// parallel with the rest of the library).
#include "shapes.h"

namespace adscl {

// id, P, NT, CL
#define ADSCL_SHAPES(X)                                                                  \
    X(0, 8, 512, 1) X(1, 8, 512, 2) X(2, 8, 512, 4) X(3, 8, 512, 8)                      \
    X(4, 4, 512, 1) X(5, 4, 512, 2)                                                      \
    X(6, 8, 256, 1) X(7, 8, 256, 2) X(8, 8, 256, 4)                                      \
    X(9, 4, 256, 1) X(10, 4, 256, 2) X(11, 4, 256, 4)                                    \
    X(12, 8, 128, 1) X(13, 4, 128, 1) X(14, 8, 128, 2) X(15, 8, 128, 4)                  \
    X(16, 8, 512, 16) X(17, 8, 512, 9)

#define ADSCL_ROW(i, p, nt, cl) {p, nt, cl},
const Shape kShapes[kNumShapes] = {ADSCL_SHAPES(ADSCL_ROW)};
#undef ADSCL_ROW

int shape_index(int P, int NT, int CL)
{
    for (int i = 0; i < kNumShapes; ++i)
        if (kShapes[i].P == P && kShapes[i].NT == NT && kShapes[i].CL == CL) return i;
    return -1;
}

bool shape_fits(int id, int N)
{
    if (id < 0 || id >= kNumShapes) return false;
    const Shape &s = kShapes[id];
    const int T = (N - 1) / s.P;   // node blocks (N - 1 is a multiple of 8)
    return (long long)s.P * s.NT * s.CL >= N - 1 && T >= s.CL && (T + s.CL - 1) / s.CL <= s.NT;
}

namespace {

template <int P>
int stride_p(int Nloc) { return field_stride<P>(Nloc); }

// largest local node index + 1 of any CTA of the shape for grids up to Nmax
int local_nodes(int id, int Nmax)
{
    const Shape &s = kShapes[id];
    const int T = (Nmax - 1) / s.P;
    return ((T + s.CL - 1) / s.CL) * s.P + 1;
}

template <int P, int NT, int CL, bool REC>
const void *kernel_ptr() { return (const void *)evolve_kernel<P, NT, CL, REC>; }

// the kernel of shape id; rec: the variant writing the adjoint's stage record
const void *kernel_of(int id, bool rec)
{
    switch (id) {
#define ADSCL_CASE(i, p, nt, cl) case i: return rec ? kernel_ptr<p, nt, cl, true>() : kernel_ptr<p, nt, cl, false>();
        ADSCL_SHAPES(ADSCL_CASE)
#undef ADSCL_CASE
    }
    return nullptr;
}

template <int P, int NT, int CL, bool REC>
cudaError_t launch_t(const EvolveArgs &a, int units, size_t smem, int stride, cudaStream_t stream)
{
    if constexpr (CL == 1) {
        evolve_kernel<P, NT, 1, REC><<<units, NT, smem, stream>>>(a, stride);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(CL * units, 1, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, evolve_kernel<P, NT, CL, REC>, a, stride);
    }
}

}  // namespace

int shape_stride(int id, int Nmax)
{
    const int nl = local_nodes(id, Nmax);
    return kShapes[id].P == 8 ? stride_p<8>(nl) : stride_p<4>(nl);
}

size_t shape_smem(int id, int Nmax) { return (size_t)6 * shape_stride(id, Nmax) * sizeof(double); }

cudaError_t shapes_set_attributes()
{
    for (int id = 0; id < kNumShapes; ++id) {
        const Shape &s = kShapes[id];
        // the largest grid a CTA of this shape can hold: P * NT nodes (+ the closing node)
        const size_t smem = shape_smem(id, s.P * s.NT * s.CL + 1);
        for (int rec = 0; rec < 2; ++rec) {
            cudaError_t e = cudaFuncSetAttribute(kernel_of(id, rec != 0),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess && s.CL > 8)   // 9 or 16 CTAs: beyond the portable cluster size
                e = cudaFuncSetAttribute(kernel_of(id, rec != 0), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t shape_max_units(int id, size_t smem, int num_sms, int *units)
{
    const Shape &s = kShapes[id];
    *units = 0;
    if (s.CL == 1) {
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(id, false), s.NT, smem);
        if (e != cudaSuccess) return e;
        *units = per_sm * num_sms;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(s.CL * (num_sms / s.CL), 1, 1);
    cfg.blockDim = dim3(s.NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(units, kernel_of(id, false), &cfg);
}

cudaError_t shape_launch(int id, const EvolveArgs &a, int units, size_t smem, int stride, cudaStream_t stream)
{
    const bool rec = a.stage != nullptr;   // the same occupancy: 128 registers, same shared memory
    switch (id) {
#define ADSCL_CASE(i, p, nt, cl)                                                            \
    case i:                                                                                 \
        return rec ? launch_t<p, nt, cl, true>(a, units, smem, stride, stream)              \
                   : launch_t<p, nt, cl, false>(a, units, smem, stride, stream);
        ADSCL_SHAPES(ADSCL_CASE)
#undef ADSCL_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace adscl
