// grad_tc05.cu -- the broken gradient of every element (Sec. 2.2: grad_h U =
// (rx Dr + sx Ds, ry Dr + sy Ds) U on each element, the a2 step of the
// residual), with the operator products on the fifth-generation tensor cores
// (tcgen05) and the element tiles staged by the tensor memory accelerator.
//
// A CTA owns TE = 32 elements.  The product is batched over them as one
// matrix product per CTA,
//     D[(e, c)][n] = sum_j U[e][c][j] B[n][j],   M = 4 TE = 128 rows,
// with B = [Dr; Ds] (N = 2 NR rows, NR = Np rounded up to 8, zero rows and
// columns as padding) and K = Np rounded up to whole k-steps of 8.
//   * The FP64 state of the tile ([TE][4][Np], contiguous) arrives by one
//     cp.async.bulk.tensor 2-D copy (box 4 Np x TE) on an mbarrier.
//   * Every thread forms one row (e, c): U relative to the element's first
//     node (Dr 1 = Ds 1 = 0, so this changes nothing in exact arithmetic and
//     keeps large means out of the split), rounded to FP32 and split as
//     x_hi = TF32(x), x_lo = x - x_hi, written to shared memory in the
//     K-major layout without swizzle: core matrices of 8 rows x 16 bytes,
//     the two core matrices of an 8-element k-step 128 bytes apart, 8-row
//     groups 256 bytes apart.  B comes split the same way from the host.
//   * One thread issues, per k-step, tcgen05.mma kind::tf32 for A_hi B_hi,
//     A_hi B_lo and A_lo B_hi into one FP32 accumulator in tensor memory
//     (128 lanes x N columns), then tcgen05.commit to an mbarrier.
//   * Warp w reads lanes 32 w .. 32 w + 31 (its rows) with tcgen05.ld and
//     applies the metric terms: Ux = rx Ur + sx Us, Uy = ry Ur + sy Us.  The
//     rows are written to shared memory in the output layout (gx over the
//     consumed state tile, gy over the operand slices) and one thread stores
//     both tiles with two bulk copies (cp.async.bulk shared -> global); row
//     stores by every thread, 120 bytes apart, left the store path issuing
//     one 32-byte sector per lane.  Outputs that are not 16-byte aligned
//     take the row stores.
// Every wait is bounded; a wait that gives up raises the error flag and the
// CTA skips the rest of its work (the tensor memory it holds is released
// only once the product it issued has completed).
//
// The split products are good to about 2^-21 of sum |A||B| (the tensor core
// reads x_lo truncated to TF32), as for the mma.sync kernel.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "dg_stage.cuh"
#include "launch.h"

namespace dg {
namespace {

constexpr int TE = 32;            // elements per CTA tile
constexpr int NTH = 128;          // threads: one per row (element, field)

template <int P>
struct GradShape {
    static constexpr int Np = (P + 1) * (P + 2) / 2;
    static constexpr int NR = (Np + 7) / 8 * 8;          // rows per operator, padded
    static constexpr int N = 2 * NR;                     // [Dr; Ds]
    static constexpr int KP = NR;                        // K padded to whole k-steps
    static constexpr int KS = KP / 8;                    // k-steps
    static constexpr int TCOLS = N <= 32 ? 32 : 64;      // tensor-memory columns (power of 2 >= 32)
    // shared memory (bytes): the FP64 tile, A_hi, A_lo, B_hi, B_lo per k-step
    static constexpr size_t TILE = size_t(TE) * 4 * Np * 8;
    static constexpr size_t A_SLICE = 128 * 8 * 4;       // 4 KB: 16 row groups x 2 core matrices
    static constexpr size_t B_SLICE = size_t(N) * 8 * 4;
    static constexpr size_t oTile = 0;
    static constexpr size_t oAhi = (TILE + 1023) & ~size_t(1023);
    static constexpr size_t oAlo = oAhi + KS * A_SLICE;
    static constexpr size_t oBhi = oAlo + KS * A_SLICE;
    static constexpr size_t oBlo = oBhi + KS * B_SLICE;
    static constexpr size_t oBar = oBlo + KS * B_SLICE;   // two mbarriers (8 B each), then the tmem slot
    static constexpr size_t bytes = oBar + 32 + 1024;    // + room to align the base
    static_assert(N % 16 == 0 && N <= 256, "tcgen05 M = 128 needs N a multiple of 16");
    static_assert(2 * KS * A_SLICE >= TILE, "the gy tile is staged over the operand slices");
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

// byte offset of element (row r, k-index kk < 8) of one k-step slice in the
// K-major layout without swizzle
__host__ __device__ __forceinline__ unsigned kmajor_off(int r, int kk)
{
    return static_cast<unsigned>((r >> 3) * 256 + (kk >> 2) * 128 + (r & 7) * 16 + (kk & 3) * 4);
}

// shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (between the core matrices of a k-step), stride byte offset
// (between 8-row groups), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(unsigned addr)
{
    const uint64_t lbo = 128 >> 4, sbo = 256 >> 4;
    return (uint64_t((addr & 0x3FFFFu) >> 4)) | (lbo << 16) | (sbo << 32) | (uint64_t(1) << 46);
}

// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x)
{
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
}

// bounded wait on phase `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(64);
    }
    return false;
}

// up to p = 4 six CTAs fit an SM by shared memory; the launch bound holds
// the registers to 80 so that they do by registers too (192 -> 178 us on
// 512^2 at p = 4)
template <int P>
__global__ void __launch_bounds__(NTH, P <= 4 ? 6 : 1)
grad_tc05_kernel(const __grid_constant__ CUtensorMap tmap, const float *bimg, const double *geo, long long K,
                 double *gx, double *gy, int *err, unsigned wait_limit, int bulk_out)
{
    using S = GradShape<P>;
    constexpr int Np = S::Np, NR = S::NR, KS = S::KS;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // the layout assumes a 1024-byte aligned base (TMA destinations need 128)
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const double *tile = reinterpret_cast<const double *>(sm + S::oTile);
    float *Ahi = reinterpret_cast<float *>(sm + S::oAhi);
    float *Alo = reinterpret_cast<float *>(sm + S::oAlo);
    float *Bhi = reinterpret_cast<float *>(sm + S::oBhi);
    uint64_t *barT = reinterpret_cast<uint64_t *>(sm + S::oBar);
    uint64_t *barM = barT + 1;
    unsigned *tslot = reinterpret_cast<unsigned *>(barT + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long k0 = static_cast<long long>(blockIdx.x) * TE;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(barT)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(barM)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(unsigned(S::TCOLS))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = *tslot;

    // the tile's FP64 state: rows of 4 Np doubles, one per element (rows past K read as zero)
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(barT)),
                     "r"(unsigned(S::TILE))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(smem_u32(sm + S::oTile)), "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(int(k0)),
            "r"(smem_u32(barT))
            : "memory");
    }
    // the split operators (host image in the final layout) meanwhile
    {
        const float4 *src = reinterpret_cast<const float4 *>(bimg);
        float4 *dst = reinterpret_cast<float4 *>(Bhi);
        for (int i = tid; i < int(2 * KS * S::B_SLICE / 16); i += NTH) dst[i] = src[i];
    }
    bool ok = mbar_wait(barT, 0, wait_limit);
    // row (e, c) of A: the state relative to the element's first node, split
    const int e = tid >> 2, c = tid & 3;
    if (ok) {
        const double *u = tile + (e * 4 + c) * Np;
        const double ref = u[0];
#pragma unroll
        for (int kk = 0; kk < S::KP; ++kk) {
            // FP64 difference, narrowed with integer operations (the FP64
            // pipe of this GPU is slow; conversions run on it)
            const float x = (kk < Np) ? cvt_d2f(u[kk] - ref) : 0.f;
            const float hi = tf32_rna(x), lo = x - hi;
            const unsigned off = (kk >> 3) * unsigned(S::A_SLICE) + kmajor_off(tid, kk & 7);
            *reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(Ahi) + off) = hi;
            *reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(Alo) + off) = lo;
        }
    }
    // generic-proxy writes of A and B become visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ok = __syncthreads_and(ok);
    if (ok && tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        constexpr uint32_t idesc = idesc_tf32(128, S::N);
        const unsigned ahi = smem_u32(sm + S::oAhi), alo = smem_u32(sm + S::oAlo);
        const unsigned bhi = smem_u32(sm + S::oBhi), blo = smem_u32(sm + S::oBlo);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const uint64_t dAh = smem_desc(ahi + ks * unsigned(S::A_SLICE)), dAl = smem_desc(alo + ks * unsigned(S::A_SLICE));
            const uint64_t dBh = smem_desc(bhi + ks * unsigned(S::B_SLICE)), dBl = smem_desc(blo + ks * unsigned(S::B_SLICE));
            const uint64_t As[3] = {dAh, dAh, dAl}, Bs[3] = {dBh, dBl, dBh};
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const unsigned acc = (ks > 0 || t > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(taddr), "l"(As[t]), "l"(Bs[t]), "r"(idesc), "r"(acc)
                    : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(barM))
                     : "memory");
    }
    bool done = ok && mbar_wait(barM, 0, wait_limit);
    done = __syncthreads_and(done);
    if (done) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // this warp's 32 rows, all N columns, 16 at a time
        float d[S::N];
#pragma unroll
        for (int c0 = 0; c0 < S::N; c0 += 16) {
            unsigned r[16];
            const unsigned ta = taddr + (unsigned(warp * 32) << 16) + unsigned(c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) d[c0 + q] = __uint_as_float(r[q]);
        }
        const long long k = k0 + e;
        // bulk_out: the rows go to shared memory in the output layout -- gx
        // over the consumed state tile, gy over the operand slices, whose
        // product has completed -- and leave by two bulk copies; otherwise
        // (outputs not 16-byte aligned) every thread stores its row
        double *ox = bulk_out ? reinterpret_cast<double *>(sm + S::oTile) + (e * 4 + c) * Np : gx + (k * 4 + c) * Np;
        double *oy = bulk_out ? reinterpret_cast<double *>(sm + S::oAhi) + (e * 4 + c) * Np : gy + (k * 4 + c) * Np;
        if (k < K) {
            // metric terms in FP32 (the products are FP32-accurate), widened exactly
            const double *g = geo + k * 16;
            const float rx = cvt_d2f(g[G_RX]), ry = cvt_d2f(g[G_RY]), sx = cvt_d2f(g[G_SX]), sy = cvt_d2f(g[G_SY]);
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                const float ur = d[j], us = d[NR + j];
                ox[j] = cvt_f2d(fmaf(rx, ur, sx * us));
                oy[j] = cvt_f2d(fmaf(ry, ur, sy * us));
            }
        }
        if (bulk_out) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                const unsigned nb = static_cast<unsigned>((K - k0) < TE ? (K - k0) : TE) * 4u * Np * 8u;
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gx + k0 * 4 * Np),
                             "r"(smem_u32(sm + S::oTile)), "r"(nb)
                             : "memory");
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gy + k0 * 4 * Np),
                             "r"(smem_u32(sm + S::oAhi)), "r"(nb)
                             : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                // the copies have read shared memory before the CTA releases it
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // release the tensor memory unless a product issued here may still be running
    if (warp == 0 && (done || !ok))
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(unsigned(S::TCOLS))
                     : "memory");
}

// FP64 reference on the CUDA cores: one thread per (element, node)
template <int P>
__global__ void grad_fp64_kernel(const double *U, const double *Dr, const double *Ds, const double *geo, long long K,
                                 double *gx, double *gy)
{
    constexpr int Np = (P + 1) * (P + 2) / 2;
    const long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (n >= K * Np) return;
    const long long k = n / Np;
    const int i = static_cast<int>(n - k * Np);
    const double *g = geo + k * 16;
    const double rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double *u = U + (k * 4 + c) * Np;
        double ur = 0.0, us = 0.0;
        for (int j = 0; j < Np; ++j) {
            ur += Dr[i * Np + j] * u[j];
            us += Ds[i * Np + j] * u[j];
        }
        gx[(k * 4 + c) * Np + i] = rx * ur + sx * us;
        gy[(k * 4 + c) * Np + i] = ry * ur + sy * us;
    }
}

float tf32_round_host(float x)
{
    unsigned u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xffffe000u;          // nearest, ties away from zero
    std::memcpy(&x, &u, 4);
    return x;
}

template <int P>
cudaError_t grad_tc05_p(const GradTc05Args &a, cudaStream_t st)
{
    using S = GradShape<P>;
    constexpr int Np = S::Np;
    if (a.K < 1) return cudaSuccess;
    cudaError_t e;
    if (a.upload_ops) {
        // the split [Dr; Ds] in the kernel's shared-memory layout: hi slices, then lo slices
        std::vector<float> img(2 * S::KS * S::B_SLICE / 4, 0.f);
        for (int n = 0; n < S::N; ++n) {
            const int row = n % S::NR;
            const double *A = (n < S::NR) ? a.Dr : a.Ds;
            for (int kk = 0; kk < S::KP; ++kk) {
                const double x = (row < Np && kk < Np) ? A[row * Np + kk] : 0.0;
                const float hi = tf32_round_host(static_cast<float>(x));
                const float lo = static_cast<float>(x - static_cast<double>(hi));
                const size_t off = (kk >> 3) * S::B_SLICE + kmajor_off(n, kk & 7);
                img[off / 4] = hi;
                img[(S::KS * S::B_SLICE + off) / 4] = lo;
            }
        }
        e = cudaMemcpyAsync(a.bimg, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    // tensor map of the FP64 state: rows of 4 Np doubles, K rows; box of TE rows
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {cuuint64_t(4 * Np), cuuint64_t(a.K)};
    const cuuint64_t gstride[1] = {cuuint64_t(4 * Np) * 8};
    const cuuint32_t box[2] = {cuuint32_t(4 * Np), cuuint32_t(TE)};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(a.U), gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    auto kern = grad_tc05_kernel<P>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(S::bytes));
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>((a.K + TE - 1) / TE);
    // tile stores by bulk copies need 16-byte aligned outputs (any cudaMalloc
    // or torch allocation; tile offsets are multiples of 1 KB)
    const int bulk_out = ((reinterpret_cast<uintptr_t>(a.gx) | reinterpret_cast<uintptr_t>(a.gy)) & 15u) == 0;
    kern<<<grid, NTH, S::bytes, st>>>(tmap, a.bimg, a.geo, a.K, a.gx, a.gy, a.err, a.wait_limit, bulk_out);
    return cudaGetLastError();
}

template <int P>
cudaError_t grad_fp64_p(const GradTc05Args &a, cudaStream_t st)
{
    constexpr int Np = (P + 1) * (P + 2) / 2;
    const long long n = a.K * Np;
    if (n < 1) return cudaSuccess;
    grad_fp64_kernel<P><<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(a.U, a.Dr_dev, a.Ds_dev, a.geo,
                                                                                 a.K, a.gx, a.gy);
    return cudaGetLastError();
}

}  // namespace

size_t grad_tc05_bimg_floats(int p)
{
    const int Np = (p + 1) * (p + 2) / 2, NR = (Np + 7) / 8 * 8;
    return static_cast<size_t>(2 * (NR / 8)) * (2 * NR) * 8;
}

cudaError_t launch_broken_gradient(int p, int impl, const GradTc05Args &a, cudaStream_t st)
{
#define C_(P) (impl == 1 ? grad_tc05_p<P>(a, st) : grad_fp64_p<P>(a, st))
    switch (p) {
    case 1: return C_(1);
    case 2: return C_(2);
    case 3: return C_(3);
    case 4: return C_(4);
    case 5: return C_(5);
    case 6: return C_(6);
    default: return cudaErrorInvalidValue;
    }
#undef C_
}

}  // namespace dg
