// spectrum_tc.cuh -- the mode projections Pi_j = sum_i u_i e_j(x_i), Phi_j = sum_i v_i e_j'(x_i)
// of spectrum.cuh on the 5th-generation tensor cores (tcgen05), as dense products
//   D[instance, j] = sum_k U[instance, k] B[j, k],   128 instances x 64 modes per CTA,
// with split operands: each FP64 value is written as hi + lo (hi = the value rounded to BF16 or
// TF32, lo = the rounded remainder), and D = Uhi Bhi + (Uhi Blo + Ulo Bhi).  The two parts are
// accumulated in FP32 in two separate tensor-memory accumulators (columns 0..63: hi*hi; columns
// 64..127: the two correction products) and added in FP64 in the epilogue.
//
// Error of one projection P = sum_k u_k b_k over the K range of a task (p = 8 bits for BF16,
// 11 for TF32; L1 = sum_k |u_k b_k|):
//   - split: u = hi + lo + d with |d| <= 2^-2p |u|; the dropped terms lo*lo, hi*db, lo*db, du*b
//     add at most 3 2^-2p |u_k b_k| per term, 3 2^-2p L1 in all;
//   - accumulation: every MMA instruction adds its products to an FP32 accumulator; each such
//     accumulation is taken to err by at most one unit in the last place of the running sum
//     (2^-23 relative: the tensor cores' FP32 accumulation is not guaranteed to round to
//     nearest).  The hi*hi accumulator takes n_hh = (64 / k) accumulations per 64-element chunk
//     (k = 16 per BF16 instruction, 8 per TF32 instruction), so it errs by <= n_hh 2^-23 L1; the
//     correction accumulator holds values ~2^-p smaller and errs by <= 2 n_hh 2^{-p-23} L1.
//   One accumulator for all three products, as an earlier version had, takes 3 n_hh FP32
//   accumulations of the full-size sum per chunk; with several chunks per task that error grows
//   with the run length and dominated: it is why TF32 x3 (twice the instructions per chunk)
//   measured worse than BF16 x3 in that version.
// Split K: every task covers `chunks` 64-element K chunks of one 128 x 64 tile (1 by default,
// the shortest FP32 run) and writes its FP64 partial product; the partials of a tile are summed
// in FP64, in a fixed order, by the energy kernel.
//
// Data path per CTA (128 threads): for each 64-element K chunk the four operand tiles (U hi/lo:
// 128 rows, B hi/lo: 64 rows) are copied from global memory into shared memory in the
// no-swizzle K-major layout of 8-row x 16-byte core matrices (K-adjacent core matrices 128 B
// apart, 8-row groups kgroups * 128 B apart); one thread issues the MMAs (M = 128, N = 64,
// K = 16 for BF16 or 8 for TF32 per instruction) and commits them to an mbarrier; every thread
// waits on it (bounded) before the tiles are overwritten.  At the end each warp reads its 32
// accumulator lanes with tcgen05.ld and the CTA frees its tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace adscl {

constexpr int kTcM = 128;     // instances per CTA tile
constexpr int kTcN = 64;      // modes per CTA tile (accumulator columns)
constexpr int kTcKC = 64;     // K elements per shared-memory chunk
constexpr long long kTcSpin = 1LL << 22;

struct TcTask {
    const void *Ahi, *Alo;  // kTcM x Kpad rows of this tile (row-major, K contiguous)
    const void *Bhi, *Blo;  // kTcN x Kpad
    int Kpad;               // row length, a multiple of kTcKC
    int k0, k1;             // K chunks [k0, k1) of this task (k1 > k0)
    double *D;              // kTcM x kTcN partial product over those chunks
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t make_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: FP32 accumulator, A and B of format `fmt` (1 = BF16 for kind::f16,
// 2 = TF32 for kind::tf32), both K-major, N = kTcN, M = kTcM
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) |
           ((uint32_t)(kTcM >> 4) << 24);
}

template <bool kTf32>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
    if (kTf32) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                     :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                     :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
    return ok != 0;
}

// 16 consecutive FP32 accumulator columns of this warp's 32 lanes (completed by tcgen05.wait::ld)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

// copy rows [0, rows) x K chunk kc of a row-major operand into the core-matrix layout
template <int ES>
__device__ __forceinline__ void stage_tile(char *dst, const char *src, int rows, int Kpad, int kc) {
    constexpr int kGroups = kTcKC * ES / 16;  // 16-byte K groups per row in one chunk
    const int nvec = rows * kGroups;
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
        const int r = v / kGroups, kg = v - r * kGroups;
        const uint4 val = *reinterpret_cast<const uint4 *>(src + ((size_t)r * Kpad + (size_t)kc * kTcKC) * ES + kg * 16);
        const int off = ((r >> 3) * kGroups + kg) * 128 + (r & 7) * 16;
        *reinterpret_cast<uint4 *>(dst + off) = val;
    }
}

// one CTA per task; 128 threads; `err` receives 1 if a bounded wait ran out
template <bool kTf32>
__global__ void __launch_bounds__(128) spectrum_tc_kernel(const TcTask *tasks, int *err)
{
    constexpr int ES = kTf32 ? 4 : 2;                 // bytes per operand element
    constexpr int kGroups = kTcKC * ES / 16;
    constexpr int kStepK = 32 / ES;                   // K per MMA instruction (32 bytes)
    constexpr int kSteps = kTcKC / kStepK;
    constexpr int kABytes = kTcM * kTcKC * ES, kBBytes = kTcN * kTcKC * ES;
    constexpr uint32_t kIdesc = make_idesc(kTf32 ? 2u : 1u);
    extern __shared__ __align__(1024) char tc_smem[];
    char *sAhi = tc_smem, *sAlo = sAhi + kABytes, *sBhi = sAlo + kABytes, *sBlo = sBhi + kBBytes;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;

    const TcTask t = tasks[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_addr = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_addr) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // two accumulators of kTcN columns: hi*hi, and the corrections
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(2 * kTcN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    for (int kc = t.k0; kc < t.k1; ++kc) {
        stage_tile<ES>(sAhi, (const char *)t.Ahi, kTcM, t.Kpad, kc);
        stage_tile<ES>(sAlo, (const char *)t.Alo, kTcM, t.Kpad, kc);
        stage_tile<ES>(sBhi, (const char *)t.Bhi, kTcN, t.Kpad, kc);
        stage_tile<ES>(sBlo, (const char *)t.Blo, kTcN, t.Kpad, kc);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(sAhi), alo = smem_u32(sAlo);
            const uint32_t bhi = smem_u32(sBhi), blo = smem_u32(sBlo);
            const uint32_t sboA = kGroups * 128, sboB = kGroups * 128;
#pragma unroll
            for (int s = 0; s < kSteps; ++s) {
                const uint32_t o = s * 256;  // two K-adjacent core matrices per instruction
                const uint32_t acc0 = (kc > t.k0 || s > 0) ? 1u : 0u;
                tc_mma<kTf32>(tmem, make_smem_desc(ahi + o, 128, sboA), make_smem_desc(bhi + o, 128, sboB), kIdesc, acc0);
                tc_mma<kTf32>(tmem + kTcN, make_smem_desc(ahi + o, 128, sboA), make_smem_desc(blo + o, 128, sboB), kIdesc, acc0);
                tc_mma<kTf32>(tmem + kTcN, make_smem_desc(alo + o, 128, sboA), make_smem_desc(bhi + o, 128, sboB), kIdesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar_addr) : "memory");
        }
        // every thread waits for the MMAs before the tiles are overwritten (bounded)
        long long spin = 0;
        while (!mbar_try_wait(mbar_addr, (uint32_t)((kc - t.k0) & 1))) {
            if (++spin > kTcSpin) {
                s_fail = 1;
                break;
            }
        }
        __syncthreads();
        if (s_fail) break;
    }
    if (s_fail) {
        // give the tensor core a second bounded chance to finish before the memory is freed
        long long spin = 0;
        while (!mbar_try_wait(mbar_addr, (uint32_t)((t.k1 - t.k0 - 1) & 1)) && ++spin < kTcSpin) {}
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // warp w reads accumulator lanes 32w .. 32w+31 (= tile rows), columns 0 .. 63 of both
        // accumulators, and writes their sum in FP64
        const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16);
        double *drow = t.D + (size_t)(32 * warp + lane) * kTcN;
#pragma unroll
        for (int c = 0; c < kTcN; c += 16) {
            uint32_t r[16], q2[16];
            tc_ld16(base + c, r);
            tc_ld16(base + kTcN + c, q2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q)
                drow[c + q] = (double)__uint_as_float(r[q]) + (double)__uint_as_float(q2[q]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * kTcN) : "memory");
    }
}

// split FP64 values into hi + lo operands: BF16 (kTf32 = false) or TF32 stored as FP32 bits
template <bool kTf32>
__device__ __forceinline__ void split_value(double x, void *hi, void *lo, size_t i) {
    if (kTf32) {
        uint32_t h, l;
        const float xf = (float)x;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(xf));
        const float rf = (float)(x - (double)__uint_as_float(h));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rf));
        ((uint32_t *)hi)[i] = h;
        ((uint32_t *)lo)[i] = l;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
        ((__nv_bfloat16 *)hi)[i] = h;
        ((__nv_bfloat16 *)lo)[i] = l;
    }
}

// rows of src (row stride ld_src, length n) -> split operand rows of length Kpad (zero padded);
// grid.y = row, rows beyond nrows (tile padding) become zero
template <bool kTf32>
__global__ void split_rows_kernel(const double *src, const int64_t *row_off, int nrows, int n, int Kpad,
                                  void *hi, void *lo)
{
    const int r = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Kpad; k += gridDim.x * blockDim.x) {
        const double x = (r < nrows && k < n) ? src[row_off[r] + k] : 0.0;
        split_value<kTf32>(x, hi, lo, (size_t)r * Kpad + k);
    }
}

}  // namespace adscl
