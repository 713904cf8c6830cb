// mlp.cu -- load-surrogate MLP (include/dg_mlp.h): forward, loss, backward
// and Adam as hand-written kernels.  The matrix products use the tensor
// cores through the warp-level mma.sync m16n8k16 instruction with bfloat16
// inputs and FP32 accumulation: the layers are 64..4096 rows by 128 columns,
// far too small to fill 128-row tcgen05 tiles, and every product ends in a
// fused epilogue (bias, GELU, GELU derivative, bfloat16 rounding).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dg_mlp.h"
#include "devbuf.h"
#include "mlp_fused.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8, NTHR = 128;

enum { LAY_MK = 0, LAY_KM = 1 };          // A: [m][k] or [k][m]
enum { LAY_NK = 0, LAY_KN = 1 };          // B: [n][k] or [k][n]
enum { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DX = 2, EPI_STORE = 3 };

struct Epi {
    const float *bias;     // HIDDEN, OUT
    float *Z;              // HIDDEN: pre-activation (FP32)
    bf16 *H;               // HIDDEN: GELU(z) rounded to bfloat16
    float *Y;              // OUT: output; STORE: product
    const float *Zprev;    // DX: pre-activation of the layer below
    float *DZ32;           // DX: d loss / d z of the layer below (FP32)
    bf16 *DZ16;            // DX: the same rounded to bfloat16
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ unsigned pack2(const bf16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// C[M][N] = sum_k A(m, k) B(k, n) for bfloat16 A, B; block tile 64 x 64,
// four warps of 32 x 32 (2 x 4 mma tiles of 16 x 8), K staged by 32.
template <int ALAY, int BLAY, int EPI>
__global__ void __launch_bounds__(NTHR)
gemm_bf16_kernel(const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb, int M, int N, int K,
                 int kchunk, Epi ep)
{
    // split K: block z sums k in [z kchunk, (z + 1) kchunk); EPI_STORE writes slice z
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    __shared__ __align__(16) bf16 As[BM][BK + PAD];
    __shared__ __align__(16) bf16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += NTHR) {
            int m, k;
            if (ALAY == LAY_MK) { m = idx / BK; k = idx % BK; }
            else { k = idx / BM; m = idx % BM; }
            const int gm = m0 + m, gk = k0 + k;
            bf16 v = zero;
            if (gm < M && gk < kend) v = (ALAY == LAY_MK) ? A[static_cast<long long>(gm) * lda + gk]
                                                      : A[static_cast<long long>(gk) * lda + gm];
            As[m][k] = v;
        }
        for (int idx = tid; idx < BN * BK; idx += NTHR) {
            int n, k;
            if (BLAY == LAY_NK) { n = idx / BK; k = idx % BK; }
            else { k = idx / BN; n = idx % BN; }
            const int gn = n0 + n, gk = k0 + k;
            bf16 v = zero;
            if (gn < N && gk < kend) v = (BLAY == LAY_NK) ? B[static_cast<long long>(gn) * ldb + gk]
                                                      : B[static_cast<long long>(gk) * ldb + gn];
            Bs[n][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = pack2(&As[r][kk + 2 * t]);
                af[i][1] = pack2(&As[r + 8][kk + 2 * t]);
                af[i][2] = pack2(&As[r][kk + 2 * t + 8]);
                af[i][3] = pack2(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + g;
                bfr[j][0] = pack2(&Bs[c][kk + 2 * t]);
                bfr[j][1] = pack2(&Bs[c][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                          "r"(bfr[j][1]));
        }
        __syncthreads();
    }
    // epilogue: element (row, col) of acc[i][j][r]: row g (+8 for r >= 2), col 2t (+1 for odd r)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int gm = m0 + wm + 16 * i + g + ((r >= 2) ? 8 : 0);
                const int gn = n0 + wn + 8 * j + 2 * t + (r & 1);
                if (gm >= M || gn >= N) continue;
                const long long o = static_cast<long long>(gm) * N + gn;
                const float v = acc[i][j][r];
                if (EPI == EPI_HIDDEN) {
                    const float z = v + ep.bias[gn];
                    ep.Z[o] = z;
                    ep.H[o] = __float2bfloat16_rn(gelu_f(z));
                } else if (EPI == EPI_OUT) {
                    ep.Y[o] = v + ep.bias[gn];
                } else if (EPI == EPI_DX) {
                    const float dz = v * gelu_grad_f(ep.Zprev[o]);
                    ep.DZ32[o] = dz;
                    ep.DZ16[o] = __float2bfloat16_rn(dz);
                } else {
                    ep.Y[static_cast<long long>(blockIdx.z) * M * N + o] = v;
                }
            }
}

// sum of `splits` slices of n values (split-K partial products), fixed order
__global__ void sum_slices_kernel(const float *ws, int splits, long long n, float *out)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float a = 0.f;
        for (int z = 0; z < splits; ++z) a += ws[z * n + i];
        out[i] = a;
    }
}

__global__ void to_bf16_kernel(const float *x, long long n, bf16 *out)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        out[i] = __float2bfloat16_rn(x[i]);
}

// d loss / d y = 2 (y - t) / n and per-block sums of (y - t)^2
__global__ void loss_grad_kernel(const float *Y, const float *T, long long n, float *dz32, bf16 *dz16, float *partial)
{
    __shared__ float s[256];
    float acc = 0.f;
    const float sc = 2.0f / static_cast<float>(n);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float d = Y[i] - T[i];
        acc += d * d;
        dz32[i] = sc * d;
        dz16[i] = __float2bfloat16_rn(sc * d);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void finish_loss_kernel(const float *partial, int nb, long long n, float *out)
{
    __shared__ float s[256];
    float a = 0.f;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += partial[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / static_cast<float>(n);
}

// column sums of dz [B][N] (bias gradients): block (x, y) sums 32 columns over
// the rows of chunk y into slice y of out [gridDim.y][N]
__global__ void colsum_kernel(const float *dz, int B, int N, int rows_per_chunk, float *out)
{
    __shared__ float s[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int b0 = blockIdx.y * rows_per_chunk, b1 = min(B, b0 + rows_per_chunk);
    float a = 0.f;
    if (c < N)
        for (int b = b0 + threadIdx.y; b < b1; b += 8) a += dz[static_cast<long long>(b) * N + c];
    s[threadIdx.y][threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.y == 0 && c < N) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += s[y][threadIdx.x];
        out[static_cast<long long>(blockIdx.y) * N + c] = t;
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// Adam step with the bias corrections of step *cnt taken from bc (pairs
// bc1, bc2 per step); used when the training step is replayed from a graph
__global__ void adam_indexed_kernel(float *p, const float *g, float *m, float *v, long long n, float lr, float b1,
                                    float b2, float eps, const float *bc, const int *cnt)
{
    const int k = *cnt;
    const float bc1 = bc[2 * k], bc2 = bc[2 * k + 1];
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// hist[*cnt] = *loss (if hist), then advance the step index
__global__ void record_loss_kernel(const float *loss, float *hist, int *cnt)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (hist) hist[*cnt] = *loss;
        *cnt += 1;
    }
}

// bfloat16 copies of the weight matrices (biases stay FP32)
__global__ void weights_bf16_kernel(const float *p, const long long *woff, const long long *wlen, int nl, bf16 *wq,
                                    const long long *qoff)
{
    for (int l = 0; l < nl; ++l)
        for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < wlen[l];
             i += static_cast<long long>(gridDim.x) * blockDim.x)
            wq[qoff[l] + i] = __float2bfloat16_rn(p[woff[l] + i]);
}

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct dg_mlp {
    int n_in = 0, width = 0, depth = 0, n_out = 0, max_batch = 0, nl = 0;
    std::vector<int> din, dout;                        // per layer
    std::vector<long long> woff, boff, qoff;           // offsets in params / in the bf16 weights
    long long nparams = 0, nq = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    long long step = 0;
    dg::DevBuf<float> p, m, v, g, lossbuf, partial, ws;   // ws: split-K slices
    // training replayed from a CUDA graph: one captured Adam step, the bias
    // corrections of every step of the call, the step index, the output rows
    dg::DevBuf<float> bc, yscr;
    dg::DevBuf<int> cnt;
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[3] = {nullptr, nullptr, nullptr};
    int gkey_b = 0;
    float gkey_lr = 0.0f;
    int64_t glaunches = 0;                             // kernels in the captured step
    dg::DevBuf<bf16> wq;
    dg::DevBuf<long long> dwoff, dwlen, dqoff;
    std::vector<dg::DevBuf<float>> Z, DZ32;            // per hidden layer / per layer
    std::vector<dg::DevBuf<bf16>> H, DZ16;             // H[0] = input
    // chunked path (mlp_fused.cuh): layout, whether the network fits it and
    // is using it, the most blocks per launch, per-block gradient slices
    mlpf::Net fnet{};
    bool fused_ok = false, fused_on = false;
    int fgrid = 0;
    dg::DevBuf<float> fpart, flpart;
    dg::DevBuf<bf16> wstaged;                          // W and W^T per layer in the staging layout
    ~dg_mlp()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

dg_status mfail(dg_mlp *m, dg_status st, const std::string &msg)
{
    if (m) m->err = msg;
    return st;
}

#define M_CUDA(mm, expr)                                                                    \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) return mfail(mm, DG_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int KSPLIT_MAX = 32;

template <int AL, int BL, int EPI>
cudaError_t gemm(dg_mlp *m, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const Epi &ep)
{
    // long sums (the weight gradients sum over the batch) are split into up to
    // 32 slices of at least 256 terms, written to a workspace and added in order
    int splits = 1;
    if (EPI == EPI_STORE) splits = std::max(1, std::min(KSPLIT_MAX, K / 256));
    const int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    Epi e = ep;
    if (EPI == EPI_STORE && splits > 1) e.Y = m->ws.ptr;
    gemm_bf16_kernel<AL, BL, EPI><<<grid, NTHR, 0, m->stream>>>(A, lda, B, ldb, M, N, K, kchunk, e);
    m->launches += 1;
    if (EPI == EPI_STORE && splits > 1) {
        const long long n = static_cast<long long>(M) * N;
        sum_slices_kernel<<<static_cast<int>(std::min<long long>((n + 255) / 256, 4096)), 256, 0, m->stream>>>(
            m->ws.ptr, splits, n, ep.Y);
        m->launches += 1;
    }
    return cudaGetLastError();
}

int blocks_for(long long n) { return static_cast<int>(std::min<long long>((n + 255) / 256, 4096)); }

dg_status fused_forward(dg_mlp *m, const float *X, int B, float *Y);

// forward for B rows of X (FP32 device): fills H, Z and writes Y
dg_status forward(dg_mlp *m, const float *X, int B, float *Y)
{
    if (m->fused_on) return fused_forward(m, X, B, Y);
    const long long nx = static_cast<long long>(B) * m->n_in;
    to_bf16_kernel<<<blocks_for(nx), 256, 0, m->stream>>>(X, nx, m->H[0].ptr);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    for (int l = 0; l < m->nl; ++l) {
        Epi ep{};
        ep.bias = m->p.ptr + m->boff[l];
        const bf16 *W = m->wq.ptr + m->qoff[l];
        if (l < m->nl - 1) {
            ep.Z = m->Z[l].ptr;
            ep.H = m->H[l + 1].ptr;
            M_CUDA(m, (gemm<LAY_MK, LAY_NK, EPI_HIDDEN>(m, m->H[l].ptr, m->din[l], W, m->din[l], B, m->dout[l],
                                                       m->din[l], ep)));
        } else {
            ep.Y = Y;
            M_CUDA(m, (gemm<LAY_MK, LAY_NK, EPI_OUT>(m, m->H[l].ptr, m->din[l], W, m->din[l], B, m->dout[l],
                                                    m->din[l], ep)));
        }
    }
    return DG_OK;
}

// loss and gradient (into grad) for the rows of X, T; forward included
dg_status loss_grad(dg_mlp *m, const float *X, const float *T, int B, float *grad, float *loss, float *Yscratch)
{
    dg_status st = forward(m, X, B, Yscratch);
    if (st != DG_OK) return st;
    const int L = m->nl;
    const long long ny = static_cast<long long>(B) * m->n_out;
    const int nb = std::min(blocks_for(ny), 256);
    loss_grad_kernel<<<nb, 256, 0, m->stream>>>(Yscratch, T, ny, m->DZ32[L - 1].ptr, m->DZ16[L - 1].ptr,
                                                m->partial.ptr);
    finish_loss_kernel<<<1, 256, 0, m->stream>>>(m->partial.ptr, nb, ny, loss);
    m->launches += 2;
    M_CUDA(m, cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int ni = m->din[l], no = m->dout[l];
        // dW_l = dZ_l^T H_l  (sum over the batch)
        Epi eg{};
        eg.Y = grad + m->woff[l];
        M_CUDA(m, (gemm<LAY_KM, LAY_KN, EPI_STORE>(m, m->DZ16[l].ptr, no, m->H[l].ptr, ni, no, ni, B, eg)));
        {
            const int chunks = std::max(1, std::min(KSPLIT_MAX, B / 128));
            const int rows = (B + chunks - 1) / chunks;
            colsum_kernel<<<dim3((no + 31) / 32, chunks), dim3(32, 8), 0, m->stream>>>(m->DZ32[l].ptr, B, no, rows,
                                                                                      m->ws.ptr);
            sum_slices_kernel<<<(no + 255) / 256, 256, 0, m->stream>>>(m->ws.ptr, chunks, no, grad + m->boff[l]);
            m->launches += 2;
        }
        M_CUDA(m, cudaGetLastError());
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
            Epi ed{};
            ed.Zprev = m->Z[l - 1].ptr;
            ed.DZ32 = m->DZ32[l - 1].ptr;
            ed.DZ16 = m->DZ16[l - 1].ptr;
            M_CUDA(m, (gemm<LAY_MK, LAY_KN, EPI_DX>(m, m->DZ16[l].ptr, no, m->wq.ptr + m->qoff[l], ni, B, ni, no, ed)));
        }
    }
    return DG_OK;
}

// ---- chunked path: every block takes whole 32-row chunks of the batch

int fused_blocks(const dg_mlp *m, int B) { return std::min((B + mlpf::R - 1) / mlpf::R, m->fgrid); }

int reduce_blocks(const dg_mlp *m) { return static_cast<int>((m->nparams + mlpf::RP - 1) / mlpf::RP); }

dg_status fused_forward(dg_mlp *m, const float *X, int B, float *Y)
{
    mlpf::mlp_chunk_kernel<false><<<fused_blocks(m, B), mlpf::NT, m->fnet.bytes, m->stream>>>(
        m->fnet, m->p.ptr, m->wstaged.ptr, X, nullptr, B, Y, nullptr, nullptr, nullptr);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

// gradient slices and loss sums of every block for the rows of X, T;
// step (or null): the replayed step's index, advanced by the kernel
dg_status fused_chunks(dg_mlp *m, const float *X, const float *T, int B, int *step = nullptr)
{
    mlpf::mlp_chunk_kernel<true><<<fused_blocks(m, B), mlpf::NT, m->fnet.bytes, m->stream>>>(
        m->fnet, m->p.ptr, m->wstaged.ptr, X, T, B, nullptr, m->fpart.ptr, m->flpart.ptr, step);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

dg_status fused_loss_grad(dg_mlp *m, const float *X, const float *T, int B, float *grad, float *loss)
{
    dg_status st = fused_chunks(m, X, T, B);
    if (st != DG_OK) return st;
    mlpf::mlp_reduce_kernel<false><<<reduce_blocks(m), mlpf::RP * mlpf::RQ, 0, m->stream>>>(
        m->fnet, fused_blocks(m, B), m->fpart.ptr, m->flpart.ptr, static_cast<long long>(B) * m->n_out, grad, loss,
        nullptr, nullptr, nullptr, nullptr, nullptr, mlpf::Adam{});
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

// one Adam step: loss (before the update) to *loss; bias corrections bc1,
// bc2 -- or, when bc is set (graph replay), those of step *cnt, which the
// chunk kernel advances, with the loss also written to hist[*cnt] if hist
dg_status fused_step(dg_mlp *m, const float *X, const float *T, int B, float *loss, float lr, float bc1, float bc2,
                     const float *bc, int *cnt, float *hist)
{
    dg_status st = fused_chunks(m, X, T, B, bc ? cnt : nullptr);
    if (st != DG_OK) return st;
    const mlpf::Adam o{lr, 0.9f, 0.999f, 1e-8f, bc1, bc2, bc, cnt, hist};
    mlpf::mlp_reduce_kernel<true><<<reduce_blocks(m), mlpf::RP * mlpf::RQ, 0, m->stream>>>(
        m->fnet, fused_blocks(m, B), m->fpart.ptr, m->flpart.ptr, static_cast<long long>(B) * m->n_out, nullptr,
        loss, m->p.ptr, m->m.ptr, m->v.ptr, m->wstaged.ptr, m->wq.ptr, o);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

dg_status refresh_bf16(dg_mlp *m)
{
    weights_bf16_kernel<<<blocks_for(m->nq), 256, 0, m->stream>>>(m->p.ptr, m->dwoff.ptr, m->dwlen.ptr, m->nl,
                                                                 m->wq.ptr, m->dqoff.ptr);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

// the chunked path's staged weight copies from the FP32 parameters
dg_status refresh_staged(dg_mlp *m)
{
    if (!m->fused_ok) return DG_OK;
    mlpf::mlp_stage_copies_kernel<<<blocks_for(m->nparams), 256, 0, m->stream>>>(m->fnet, m->p.ptr,
                                                                                m->wstaged.ptr);
    m->launches += 1;
    M_CUDA(m, cudaGetLastError());
    return DG_OK;
}

dg_status check_rows(dg_mlp *m, const void *a, const void *b, int B)
{
    if (!a || !b) return mfail(m, DG_EINVAL, "null device array");
    if (B < 1 || B > m->max_batch) return mfail(m, DG_EINVAL, "batch size out of range");
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_mlp_create(int n_in, int width, int depth, int n_out, int max_batch, uint64_t seed, dg_mlp **out)
{
    if (!out) return DG_EINVAL;
    *out = nullptr;
    if (n_in < 1 || width < 1 || depth < 1 || n_out < 1 || max_batch < 1 || width > 4096 || n_in > 4096 ||
        n_out > 4096 || max_batch > (1 << 20))
        return DG_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return DG_ECUDA;
    }
    dg_mlp *m = new dg_mlp();
    m->n_in = n_in;
    m->width = width;
    m->depth = depth;
    m->n_out = n_out;
    m->max_batch = max_batch;
    m->nl = depth + 1;
    for (int l = 0; l < m->nl; ++l) {
        m->din.push_back(l == 0 ? n_in : width);
        m->dout.push_back(l == m->nl - 1 ? n_out : width);
    }
    long long o = 0, q = 0;
    std::vector<long long> wlen;
    for (int l = 0; l < m->nl; ++l) {
        m->woff.push_back(o);
        m->qoff.push_back(q);
        wlen.push_back(static_cast<long long>(m->din[l]) * m->dout[l]);
        o += wlen.back();
        q += wlen.back();
        m->boff.push_back(o);
        o += m->dout[l];
    }
    m->nparams = o;
    m->nq = q;
    // seeded init
    std::vector<float> h(static_cast<size_t>(o), 0.0f);
    uint64_t s = seed;
    for (int l = 0; l < m->nl; ++l) {
        const double a = std::sqrt(6.0 / (m->din[l] + m->dout[l]));
        for (long long i = 0; i < wlen[l]; ++i) {
            const double u = static_cast<double>(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            h[m->woff[l] + i] = static_cast<float>((2.0 * u - 1.0) * a);
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    chk(m->p.alloc(o));
    chk(m->m.alloc(o));
    chk(m->v.alloc(o));
    chk(m->g.alloc(o));
    chk(m->wq.alloc(q));
    chk(m->lossbuf.alloc(1));
    chk(m->partial.alloc(256));
    {
        long long mx = 0;
        for (int l = 0; l < m->nl; ++l) mx = std::max(mx, static_cast<long long>(m->din[l]) * m->dout[l]);
        chk(m->ws.alloc(static_cast<size_t>(mx) * KSPLIT_MAX));
    }
    chk(m->dwoff.alloc(m->nl));
    chk(m->dwlen.alloc(m->nl));
    chk(m->dqoff.alloc(m->nl));
    m->Z.resize(m->nl);
    m->H.resize(m->nl);
    m->DZ32.resize(m->nl);
    m->DZ16.resize(m->nl);
    const long long mb = max_batch;
    chk(m->H[0].alloc(static_cast<size_t>(mb * n_in)));
    for (int l = 0; l < m->nl; ++l) {
        if (l < m->nl - 1) {
            chk(m->Z[l].alloc(static_cast<size_t>(mb * m->dout[l])));
            chk(m->H[l + 1].alloc(static_cast<size_t>(mb * m->dout[l])));
        }
        chk(m->DZ32[l].alloc(static_cast<size_t>(mb * m->dout[l])));
        chk(m->DZ16[l].alloc(static_cast<size_t>(mb * m->dout[l])));
    }
    if (e == cudaSuccess) {
        chk(cudaMemcpy(m->p.ptr, h.data(), o * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemset(m->m.ptr, 0, o * sizeof(float)));
        chk(cudaMemset(m->v.ptr, 0, o * sizeof(float)));
        chk(cudaMemcpy(m->dwoff.ptr, m->woff.data(), m->nl * sizeof(long long), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(m->dwlen.ptr, wlen.data(), m->nl * sizeof(long long), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(m->dqoff.ptr, m->qoff.data(), m->nl * sizeof(long long), cudaMemcpyHostToDevice));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return DG_ECUDA;
    }
    {
        // the chunked path, if the layers fit a block's shared memory
        int dev = 0, smax = 0, sms = 0;
        chk(cudaGetDevice(&dev));
        chk(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        chk(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (e == cudaSuccess && mlpf::plan(m->fnet, m->nl, m->din.data(), m->dout.data(), m->woff.data(),
                                           m->boff.data(), m->qoff.data(), m->nparams, static_cast<size_t>(smax))) {
            const int bytes = static_cast<int>(m->fnet.bytes);
            chk(cudaFuncSetAttribute(mlpf::mlp_chunk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            chk(cudaFuncSetAttribute(mlpf::mlp_chunk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            m->fgrid = std::max(1, std::min(sms, (max_batch + mlpf::R - 1) / mlpf::R));
            chk(m->fpart.alloc(static_cast<size_t>(m->fgrid) * static_cast<size_t>(m->nparams)));
            chk(m->flpart.alloc(static_cast<size_t>(m->fgrid)));
            chk(m->wstaged.alloc(static_cast<size_t>(m->fnet.nstaged)));
            if (e == cudaSuccess) chk(cudaMemset(m->wstaged.ptr, 0, sizeof(bf16) * m->fnet.nstaged));
            m->fused_ok = m->fused_on = (e == cudaSuccess);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return DG_ECUDA;
    }
    if (refresh_bf16(m) != DG_OK || refresh_staged(m) != DG_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return DG_ECUDA;
    }
    *out = m;
    return DG_OK;
}

dg_status dg_mlp_destroy(dg_mlp *m)
{
    delete m;
    return DG_OK;
}

const char *dg_mlp_last_error(const dg_mlp *m) { return m ? m->err.c_str() : "null network"; }

int64_t dg_mlp_param_count(const dg_mlp *m) { return m ? m->nparams : 0; }

int64_t dg_mlp_kernel_launches(const dg_mlp *m) { return m ? m->launches : 0; }

dg_status dg_mlp_set_params(dg_mlp *m, const float *params, int on_device)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    if (!params) return mfail(m, DG_EINVAL, "null parameters");
    M_CUDA(m, cudaMemcpyAsync(m->p.ptr, params, m->nparams * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    M_CUDA(m, cudaMemsetAsync(m->m.ptr, 0, m->nparams * sizeof(float), m->stream));
    M_CUDA(m, cudaMemsetAsync(m->v.ptr, 0, m->nparams * sizeof(float), m->stream));
    m->step = 0;
    dg_status st = refresh_bf16(m);
    if (st == DG_OK) st = refresh_staged(m);
    if (st != DG_OK) return st;
    M_CUDA(m, cudaStreamSynchronize(m->stream));
    return DG_OK;
}

dg_status dg_mlp_get_params(dg_mlp *m, float *params, int on_device)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    if (!params) return mfail(m, DG_EINVAL, "null parameters");
    M_CUDA(m, cudaMemcpyAsync(params, m->p.ptr, m->nparams * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
    M_CUDA(m, cudaStreamSynchronize(m->stream));
    return DG_OK;
}

dg_status dg_mlp_set_fused(dg_mlp *m, int on)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    if (on && !m->fused_ok) return mfail(m, DG_EUNSUPPORTED, "the layers do not fit the chunked path");
    if ((on != 0) == m->fused_on) return DG_OK;
    if (m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    m->fused_on = on != 0;
    if (m->fused_on) {
        // the layer-by-layer kernels keep only the row-major bf16 copy current
        dg_status st = refresh_staged(m);
        if (st != DG_OK) return st;
        M_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    return DG_OK;
}

int dg_mlp_is_fused(const dg_mlp *m) { return (m && m->fused_on) ? 1 : 0; }

dg_status dg_mlp_forward(dg_mlp *m, const float *X, int B, float *Y)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    dg_status st = check_rows(m, X, Y, B);
    if (st != DG_OK) return st;
    st = forward(m, X, B, Y);
    if (st != DG_OK) return st;
    M_CUDA(m, cudaStreamSynchronize(m->stream));
    return DG_OK;
}

dg_status dg_mlp_loss_grad(dg_mlp *m, const float *X, const float *T, int B, float *grad, float *loss)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    dg_status st = check_rows(m, X, T, B);
    if (st != DG_OK) return st;
    if (!grad || !loss) return mfail(m, DG_EINVAL, "null output");
    if (m->fused_on) {
        st = fused_loss_grad(m, X, T, B, grad, loss);
    } else {
        dg::DevBuf<float> y;
        M_CUDA(m, y.alloc(static_cast<size_t>(B) * m->n_out));
        st = loss_grad(m, X, T, B, grad, loss, y.ptr);
    }
    if (st != DG_OK) return st;
    M_CUDA(m, cudaStreamSynchronize(m->stream));
    return DG_OK;
}

dg_status dg_mlp_train(dg_mlp *m, const float *X, const float *T, int B, int nsteps, float lr, float *loss_hist)
{
    if (!m) return DG_EINVAL;
    m->err.clear();
    dg_status st = check_rows(m, X, T, B);
    if (st != DG_OK) return st;
    if (nsteps < 0 || !(lr > 0.0f)) return mfail(m, DG_EINVAL, "need nsteps >= 0 and lr > 0");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    if (!m->yscr.ptr) M_CUDA(m, m->yscr.alloc(static_cast<size_t>(m->max_batch) * m->n_out));
    if (nsteps < 8) {
        for (int n = 0; n < nsteps; ++n) {
            float *lo = loss_hist ? loss_hist + n : m->lossbuf.ptr;
            const float bc1 = static_cast<float>(1.0 - std::pow(0.9, static_cast<double>(m->step + 1)));
            const float bc2 = static_cast<float>(1.0 - std::pow(0.999, static_cast<double>(m->step + 1)));
            if (m->fused_on) {
                st = fused_step(m, X, T, B, lo, lr, bc1, bc2, nullptr, nullptr, nullptr);
                if (st != DG_OK) return st;
                m->step += 1;
                continue;
            }
            st = loss_grad(m, X, T, B, m->g.ptr, lo, m->yscr.ptr);
            if (st != DG_OK) return st;
            m->step += 1;
            adam_kernel<<<blocks_for(m->nparams), 256, 0, m->stream>>>(m->p.ptr, m->g.ptr, m->m.ptr, m->v.ptr,
                                                                      m->nparams, lr, b1, b2, eps, bc1, bc2);
            m->launches += 1;
            M_CUDA(m, cudaGetLastError());
            st = refresh_bf16(m);
            if (st != DG_OK) return st;
        }
        M_CUDA(m, cudaStreamSynchronize(m->stream));
        return DG_OK;
    }
    // Longer runs replay one captured step: the same kernels with the same
    // arguments as above, the bias corrections (computed here in double, as
    // above) and the loss history indexed by a device step counter.
    std::vector<float> bch(2 * static_cast<size_t>(nsteps));
    for (int n = 0; n < nsteps; ++n) {
        const double k = static_cast<double>(m->step + 1 + n);
        bch[2 * n] = static_cast<float>(1.0 - std::pow(0.9, k));
        bch[2 * n + 1] = static_cast<float>(1.0 - std::pow(0.999, k));
    }
    if (m->bc.n < bch.size()) {
        if (m->gexec) {
            cudaGraphExecDestroy(m->gexec);
            m->gexec = nullptr;
        }
        M_CUDA(m, m->bc.alloc(bch.size()));
    }
    if (!m->cnt.ptr) M_CUDA(m, m->cnt.alloc(1));
    M_CUDA(m, cudaMemcpyAsync(m->bc.ptr, bch.data(), bch.size() * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    // the step index: the chunked step advances it at its start (from -1),
    // the layer-by-layer step after its update (from 0)
    M_CUDA(m, cudaMemsetAsync(m->cnt.ptr, m->fused_on ? 0xff : 0, sizeof(int), m->stream));
    const bool same = m->gexec && m->gkey[0] == X && m->gkey[1] == T && m->gkey[2] == loss_hist && m->gkey_b == B &&
                      m->gkey_lr == lr;
    if (!same) {
        if (m->gexec) {
            cudaGraphExecDestroy(m->gexec);
            m->gexec = nullptr;
        }
        const int64_t l0 = m->launches;
        M_CUDA(m, cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
        if (m->fused_on) {
            st = fused_step(m, X, T, B, m->lossbuf.ptr, lr, 1.0f, 1.0f, m->bc.ptr, m->cnt.ptr, loss_hist);
        } else {
            st = loss_grad(m, X, T, B, m->g.ptr, m->lossbuf.ptr, m->yscr.ptr);
            adam_indexed_kernel<<<blocks_for(m->nparams), 256, 0, m->stream>>>(m->p.ptr, m->g.ptr, m->m.ptr,
                                                                              m->v.ptr, m->nparams, lr, b1, b2, eps,
                                                                              m->bc.ptr, m->cnt.ptr);
            record_loss_kernel<<<1, 32, 0, m->stream>>>(m->lossbuf.ptr, loss_hist, m->cnt.ptr);
            m->launches += 2;
            if (st == DG_OK) st = refresh_bf16(m);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(m->stream, &graph);
        if (st != DG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        M_CUDA(m, ec);
        const cudaError_t ei = cudaGraphInstantiate(&m->gexec, graph, 0);
        cudaGraphDestroy(graph);
        M_CUDA(m, ei);
        m->glaunches = m->launches - l0;
        m->launches = l0;
        m->gkey[0] = X;
        m->gkey[1] = T;
        m->gkey[2] = loss_hist;
        m->gkey_b = B;
        m->gkey_lr = lr;
    }
    for (int n = 0; n < nsteps; ++n) M_CUDA(m, cudaGraphLaunch(m->gexec, m->stream));
    m->launches += m->glaunches * nsteps;
    m->step += nsteps;
    M_CUDA(m, cudaStreamSynchronize(m->stream));
    return DG_OK;
}

}  // extern "C"
