// mlp_fused.cuh -- one training step of the surrogate network in two
// kernels, for networks whose layers fit a block's shared memory (inputs and
// hidden width <= 128, outputs <= 16, at most 8 layers).
//
// mlp_chunk_kernel: every block carries chunks of R = 32 batch rows through
// the forward pass, the loss and the backward pass.  All activations of a
// chunk stay in shared memory.  The weights are staged there one layer at a
// time, in the orientation the product needs, from two bf16 copies kept in
// global memory in exactly the shared-memory layout (W and W^T, rows padded
// with zeros); the copy for the next product is in flight (cp.async) while
// the current one runs, when two staging buffers fit.
// The products are block-wide sums of warp tiles of mma.sync m16n8k16 (bf16
// in, FP32 accumulation), with the same rounding points as the layer-by-layer
// kernels: bf16 inputs and activations, FP32 pre-activations, dz in FP32 and
// rounded to bf16 for the next products.  The block's weight and bias
// gradients over its chunks go to its own slice of a workspace, its loss sum
// to one float.
//
// mlp_reduce_kernel: adds the slices in block order (deterministic) and
// either returns the gradient and the loss or applies Adam and refreshes the
// bf16 copy of the weights.
#pragma once
#include <cuda_bf16.h>

namespace mlpf {

using bf16 = __nv_bfloat16;

constexpr int R = 32;          // batch rows per chunk
constexpr int NT = 256;        // threads per block (8 warps)
constexpr int MAXW = 128;      // largest input or hidden width
constexpr int MAXO = 16;       // largest output width
constexpr int MAXL = 8;        // most layers (hidden and output)

__host__ __device__ constexpr int kpad(int d) { return (d + 15) & ~15; }   // extent as a K dimension (16-steps)
__host__ __device__ constexpr int npad(int d) { return (d + 7) & ~7; }     // extent as an N dimension (8-tiles)
// row stride in bf16 elements of a K-contiguous operand: 8 elements past the
// K extent, so the 8 rows x 4 column pairs of a fragment load fall in 32
// distinct banks for every K extent that is a multiple of 16
__host__ __device__ constexpr int ldk(int d) { return kpad(d) + 8; }

// sizes, parameter offsets and the shared-memory layout (byte offsets)
struct Net {
    int nl, maxd;                           // layers; widest layer output
    int din[MAXL], dout[MAXL];
    long long woff[MAXL], boff[MAXL], qoff[MAXL];
    long long nparams;
    unsigned oH[MAXL];                      // bf16 [R][ldk(din[l])]: input of layer l
    unsigned oZ[MAXL];                      // float [R][dout[l]]: pre-activation of hidden layer l
    long long fo[MAXL], to[MAXL];           // element offsets of the staged copies of W_l and W_l^T
    long long nstaged;                      // elements in the two copies
    int nbuf;                               // staging buffers (2: the next copy is prefetched)
    unsigned oW[2];                         // bf16: staged weight matrices
    unsigned oB;                            // float [nl][maxd]: biases
    unsigned oD16[2];                       // bf16 [R][ldk(maxd)]: dz rounded, two buffers
    unsigned oD32;                          // float [R][maxd]: dz
    unsigned oTt, oHt;                      // bf16 [.][ldk(R)]: dz and H transposed
    unsigned oRed;                          // float [NT / 32]
    unsigned bytes;
};

// Fills the layout; false if the network does not fit this path.
inline bool plan(Net &n, int nl, const int *din, const int *dout, const long long *woff, const long long *boff,
                 const long long *qoff, long long nparams, size_t smem_max)
{
    if (nl < 2 || nl > MAXL) return false;
    n = Net{};
    n.nl = nl;
    n.nparams = nparams;
    int maxd = 0, maxi = 0;
    for (int l = 0; l < nl; ++l) {
        if (din[l] < 1 || din[l] > MAXW || dout[l] < 1) return false;
        if (l < nl - 1 ? dout[l] > MAXW : dout[l] > MAXO) return false;
        n.din[l] = din[l];
        n.dout[l] = dout[l];
        n.woff[l] = woff[l];
        n.boff[l] = boff[l];
        n.qoff[l] = qoff[l];
        maxd = dout[l] > maxd ? dout[l] : maxd;
        maxi = din[l] > maxi ? din[l] : maxi;
    }
    n.maxd = maxd;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 15) & ~size_t(15);
        return static_cast<unsigned>(o);
    };
    size_t wsz = 0;
    long long st = 0;
    for (int l = 0; l < nl; ++l) {
        n.oH[l] = take(sizeof(bf16) * R * ldk(din[l]));
        if (l < nl - 1) n.oZ[l] = take(sizeof(float) * R * dout[l]);
        const size_t fw = static_cast<size_t>(npad(dout[l])) * ldk(din[l]);     // forward: W as [n][k]
        const size_t bw = static_cast<size_t>(npad(din[l])) * ldk(dout[l]);     // backward: W^T as [n][k]
        wsz = fw > wsz ? fw : wsz;
        wsz = bw > wsz ? bw : wsz;
        n.fo[l] = st;
        st += static_cast<long long>(fw);
        n.to[l] = st;
        st += static_cast<long long>(bw);
    }
    n.nstaged = st;
    n.oB = take(sizeof(float) * nl * maxd);
    n.oW[0] = take(sizeof(bf16) * wsz);
    n.oD16[0] = take(sizeof(bf16) * R * ldk(maxd));
    n.oD16[1] = take(sizeof(bf16) * R * ldk(maxd));
    n.oD32 = take(sizeof(float) * R * maxd);
    n.oTt = take(sizeof(bf16) * kpad(maxd) * ldk(R));
    n.oHt = take(sizeof(bf16) * npad(maxi) * ldk(R));
    n.oRed = take(sizeof(float) * (NT / 32));
    // a second staging buffer if it fits
    n.nbuf = 1;
    n.oW[1] = n.oW[0];
    if (off + ((sizeof(bf16) * wsz + 15) & ~size_t(15)) <= smem_max) {
        n.oW[1] = take(sizeof(bf16) * wsz);
        n.nbuf = 2;
    }
    n.bytes = static_cast<unsigned>(off);
    return off <= smem_max;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ unsigned ld2(const bf16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// Block-wide C = A B^T over shared-memory operands: A [16 Mt][lda] and
// B [8 Nt][ldb], both K-contiguous with K = 16 Ks (zero-padded).  Each warp
// takes a 16-row strip of up to four 8-column tiles at a time and hands every
// result to epi(row, col, value).
template <typename Epi>
__device__ __forceinline__ void bgemm(const bf16 *A, int lda, const bf16 *B, int ldb, int Mt, int Nt, int Ks, Epi epi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int Nq = (Nt + 3) >> 2;
    for (int job = warp; job < Mt * Nq; job += NT / 32) {
        const int mt = job / Nq, nq = job - (job / Nq) * Nq;
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
        for (int ks = 0; ks < Ks; ++ks) {
            const bf16 *a = A + (16 * mt + g) * lda + 16 * ks + 2 * t;
            const unsigned a0 = ld2(a), a1 = ld2(a + 8 * lda), a2 = ld2(a + 8), a3 = ld2(a + 8 * lda + 8);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int nt = 4 * nq + j;
                if (nt < Nt) {
                    const bf16 *b = B + (8 * nt + g) * ldb + 16 * ks + 2 * t;
                    const unsigned b0 = ld2(b), b1 = ld2(b + 8);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                }
            }
        }
        // acc[j][r]: row g (+ 8 for r >= 2), column 2 t (+ 1 for odd r) of tile 4 nq + j
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nt = 4 * nq + j;
            if (nt < Nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) epi(16 * mt + g + ((r >= 2) ? 8 : 0), 8 * nt + 2 * t + (r & 1), acc[j][r]);
        }
    }
}

// Staging step s of a chunk: s < nl is layer s of the forward pass (W),
// s >= nl is layer 2 nl - 1 - s of the backward pass (W^T); with the block's
// copies as 16-byte cp.async into Ws, committed as one group per thread.
__device__ __forceinline__ void stage_async(const Net &net, int s, bf16 *Ws, const bf16 *__restrict__ WS)
{
    const int l = s < net.nl ? s : 2 * net.nl - 1 - s;
    const long long o = s < net.nl ? net.fo[l] : net.to[l];
    const int n = s < net.nl ? npad(net.dout[l]) * ldk(net.din[l]) : npad(net.din[l]) * ldk(net.dout[l]);
    const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(Ws));
    const bf16 *src = WS + o;
    for (int i = threadIdx.x; i < (n >> 3); i += NT)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * i), "l"(src + 8 * i));
    asm volatile("cp.async.commit_group;\n" ::);
}

// zero columns [c0, c1) of the R rows of a bf16 [R][ls] buffer
__device__ __forceinline__ void zero_cols(bf16 *D, int ls, int c0, int c1)
{
    const int w = c1 - c0;
    if (w <= 0) return;
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (int i = threadIdx.x; i < R * w; i += NT) D[(i / w) * ls + c0 + i - (i / w) * w] = zero;
}

// TRAIN = false: forward only, Y [B][n_out].  TRAIN = true: loss and
// gradient; the block's slice of part [gridDim.x][nparams] and lpart
// [gridDim.x] receive its sums over its chunks.
template <bool TRAIN>
__global__ void __launch_bounds__(NT) mlp_chunk_kernel(Net net, const float *__restrict__ P, const bf16 *__restrict__ WS,
                                                       const float *__restrict__ X, const float *__restrict__ T, int B,
                                                       float *__restrict__ Y, float *__restrict__ part,
                                                       float *__restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x;
    const int nl = net.nl, n_in = net.din[0], n_out = net.dout[nl - 1], maxd = net.maxd, LDD = ldk(maxd);
    float *D32 = reinterpret_cast<float *>(sm + net.oD32);
    bf16 *Tt = reinterpret_cast<bf16 *>(sm + net.oTt);
    bf16 *Ht = reinterpret_cast<bf16 *>(sm + net.oHt);
    const bf16 zero = __float2bfloat16_rn(0.f);
    const long long NP = net.nparams;
    const float sc = 2.0f / static_cast<float>(static_cast<long long>(B) * n_out);
    // the padding columns of the hidden activations are never written: clear once
    for (int l = 1; l < nl; ++l) zero_cols(reinterpret_cast<bf16 *>(sm + net.oH[l]), ldk(net.din[l]), net.din[l],
                                            kpad(net.din[l]));
    float *sB = reinterpret_cast<float *>(sm + net.oB);
    for (int l = 0; l < nl; ++l)
        for (int c = tid; c < net.dout[l]; c += NT) sB[l * maxd + c] = P[net.boff[l] + c];
    // weight staging: S steps per chunk, step gs (counted over the block's
    // chunks) in buffer gs % nbuf; with two buffers the next step's copy is
    // issued before the current step waits for its own
    const int S = TRAIN ? 2 * nl - 1 : nl;
    const int nchunks = (B + R - 1) / R;
    int gs = 0;
    if (net.nbuf == 2 && static_cast<int>(blockIdx.x) < nchunks)
        stage_async(net, 0, reinterpret_cast<bf16 *>(sm + net.oW[0]), WS);
    auto staged = [&](int s, int ch) -> const bf16 * {
        bf16 *cur = reinterpret_cast<bf16 *>(sm + net.oW[gs % net.nbuf]);
        if (net.nbuf == 2) {
            const bool more = s + 1 < S || ch + static_cast<int>(gridDim.x) < nchunks;
            if (more) {
                stage_async(net, (s + 1) % S, reinterpret_cast<bf16 *>(sm + net.oW[(gs + 1) & 1]), WS);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
        } else {
            stage_async(net, s, cur, WS);
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        ++gs;
        return cur;
    };
    float lacc = 0.f;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const bool first = ch == static_cast<int>(blockIdx.x);
        const int r0 = ch * R, nr = min(R, B - r0);
        {
            // layer input 0: the chunk's rows of X rounded to bf16, zero
            // outside; loads issued in groups of 8 before their stores
            bf16 *H0 = reinterpret_cast<bf16 *>(sm + net.oH[0]);
            const int kp = kpad(n_in), ls = ldk(n_in);
            for (int i0 = tid; i0 < R * kp; i0 += 8 * NT) {
                float x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * NT, r = i / kp, k = i - (i / kp) * kp;
                    x[u] = (i < R * kp && r < nr && k < n_in) ? X[static_cast<long long>(r0 + r) * n_in + k] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * NT, r = i / kp, k = i - (i / kp) * kp;
                    if (i < R * kp) H0[r * ls + k] = __float2bfloat16_rn(x[u]);
                }
            }
        }
        // ---- forward
        for (int l = 0; l < nl; ++l) {
            const int di = net.din[l], dn = net.dout[l];
            bf16 *D16 = reinterpret_cast<bf16 *>(sm + net.oD16[l & 1]);
            if (TRAIN && l == nl - 1) zero_cols(D16, LDD, dn, kpad(dn));
            const bf16 *Ws = staged(l, ch);
            __syncthreads();
            const bf16 *Hl = reinterpret_cast<const bf16 *>(sm + net.oH[l]);
            const float *bias = sB + l * maxd;
            if (l < nl - 1) {
                float *Z = reinterpret_cast<float *>(sm + net.oZ[l]);
                bf16 *Hn = reinterpret_cast<bf16 *>(sm + net.oH[l + 1]);
                const int ln = ldk(dn);
                bgemm(Hl, ldk(di), Ws, ldk(di), R / 16, npad(dn) / 8, kpad(di) / 16, [&](int r, int c, float v) {
                    if (c < dn) {
                        const float z = v + bias[c];
                        Z[r * dn + c] = z;
                        Hn[r * ln + c] = __float2bfloat16_rn(gelu(z));
                    }
                });
            } else {
                bgemm(Hl, ldk(di), Ws, ldk(di), R / 16, npad(dn) / 8, kpad(di) / 16, [&](int r, int c, float v) {
                    if (c >= dn) return;
                    const float y = v + bias[c];
                    if (!TRAIN) {
                        if (r < nr) Y[static_cast<long long>(r0 + r) * dn + c] = y;
                        return;
                    }
                    // d loss / d y of the mean squared error; rows past B add nothing
                    const float d = (r < nr) ? y - T[static_cast<long long>(r0 + r) * dn + c] : 0.f;
                    lacc += d * d;
                    D32[r * maxd + c] = sc * d;
                    D16[r * LDD + c] = __float2bfloat16_rn(sc * d);
                });
            }
            __syncthreads();
        }
        // ---- backward: layer l's gradients from dz_l, then dz_{l-1}
        for (int l = TRAIN ? nl - 1 : -1; l >= 0; --l) {
            const int di = net.din[l], dn = net.dout[l];
            const bf16 *D16 = reinterpret_cast<const bf16 *>(sm + net.oD16[l & 1]);
            const bf16 *Hl = reinterpret_cast<const bf16 *>(sm + net.oH[l]);
            float *pb = part + static_cast<long long>(blockIdx.x) * NP + net.boff[l];
            for (int c = tid; c < dn; c += NT) {
                float s = 0.f;
                for (int r = 0; r < R; ++r) s += D32[r * maxd + c];
                pb[c] = first ? s : pb[c] + s;
            }
            const int lr = ldk(R);
            for (int i = tid; i < kpad(dn) * R; i += NT) {
                const int c = i / R, r = i - (i / R) * R;
                Tt[c * lr + r] = (c < dn) ? D16[r * LDD + c] : zero;
            }
            for (int i = tid; i < npad(di) * R; i += NT) {
                const int k = i / R, r = i - (i / R) * R;
                Ht[k * lr + r] = (k < di) ? Hl[r * ldk(di) + k] : zero;
            }
            const bf16 *Ws = nullptr;
            if (l > 0) {
                bf16 *Dn = reinterpret_cast<bf16 *>(sm + net.oD16[(l - 1) & 1]);
                zero_cols(Dn, LDD, di, kpad(di));
                Ws = staged(2 * nl - 1 - l, ch);
            }
            __syncthreads();
            // dW_l += dz_l^T H_l over the chunk's rows
            float *pw = part + static_cast<long long>(blockIdx.x) * NP + net.woff[l];
            bgemm(Tt, lr, Ht, lr, kpad(dn) / 16, npad(di) / 8, R / 16, [&](int r, int c, float v) {
                if (r < dn && c < di) {
                    float *q = pw + static_cast<long long>(r) * di + c;
                    *q = first ? v : *q + v;
                }
            });
            if (l > 0) {
                // dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})
                const float *Zp = reinterpret_cast<const float *>(sm + net.oZ[l - 1]);
                bf16 *Dn = reinterpret_cast<bf16 *>(sm + net.oD16[(l - 1) & 1]);
                bgemm(D16, LDD, Ws, ldk(dn), R / 16, npad(di) / 8, kpad(dn) / 16, [&](int r, int c, float v) {
                    if (c < di) {
                        const float dz = v * gelu_grad(Zp[r * di + c]);
                        D32[r * maxd + c] = dz;
                        Dn[r * LDD + c] = __float2bfloat16_rn(dz);
                    }
                });
            }
            __syncthreads();
        }
    }
    if (TRAIN) {
        // the block's loss sum, in a fixed order
        float *red = reinterpret_cast<float *>(sm + net.oRed);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
        if ((tid & 31) == 0) red[tid >> 5] = lacc;
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            lpart[blockIdx.x] = s;
        }
    }
}

struct Adam {
    float lr, b1, b2, eps, bc1, bc2;
    const float *bc;       // if set: bias corrections (bc1, bc2) of step *cnt
    const int *cnt;
};

// weight i (a parameter index) rounded to bf16 into the staged copies WS
// (W_l at [k][n], W_l^T at [n][k]) and, if wq is set, the row-major copy
__device__ __forceinline__ void put_weight(const Net &net, long long i, float w, bf16 *WS, bf16 *wq)
{
    for (int l = 0; l < net.nl; ++l) {
        if (i < net.woff[l] || i >= net.boff[l]) continue;
        const bf16 b = __float2bfloat16_rn(w);
        const long long j = i - net.woff[l];
        const int di = net.din[l], k = static_cast<int>(j / di), n = static_cast<int>(j - (j / di) * di);
        WS[net.fo[l] + static_cast<long long>(k) * ldk(di) + n] = b;
        WS[net.to[l] + static_cast<long long>(n) * ldk(net.dout[l]) + k] = b;
        if (wq) wq[net.qoff[l] + j] = b;
    }
}

// the staged copies of every weight from the FP32 parameters (their padding
// stays as cleared at creation)
__global__ void mlp_stage_copies_kernel(Net net, const float *__restrict__ p, bf16 *WS)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < net.nparams;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        put_weight(net, i, p[i], WS, nullptr);
}

// Sum of the G slices (block order) of every parameter's gradient, and of
// the G loss sums.  ADAM = false: grad and loss out.  ADAM = true: loss out,
// Adam step on p with moments m, v, and the bf16 copies of every weight.
template <bool ADAM>
__global__ void mlp_reduce_kernel(Net net, int G, const float *__restrict__ part, const float *__restrict__ lpart,
                                  long long nsum, float *__restrict__ grad, float *__restrict__ loss, float *p, float *m,
                                  float *v, bf16 *WS, bf16 *wq, Adam o)
{
    const long long NP = net.nparams;
    float bc1 = o.bc1, bc2 = o.bc2;
    if (ADAM && o.bc) {
        const int k = *o.cnt;
        bc1 = o.bc[2 * k];
        bc2 = o.bc[2 * k + 1];
    }
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < NP;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float gi = 0.f;
        for (int c = 0; c < G; ++c) gi += part[static_cast<long long>(c) * NP + i];
        if (!ADAM) {
            grad[i] = gi;
            continue;
        }
        const float mi = o.b1 * m[i] + (1.0f - o.b1) * gi;
        const float vi = o.b2 * v[i] + (1.0f - o.b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - o.lr * (mi / bc1) / (sqrtf(vi / bc2) + o.eps);
        p[i] = pi;
        put_weight(net, i, pi, WS, wq);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int c = 0; c < G; ++c) s += lpart[c];
        *loss = s / static_cast<float>(nsum);
    }
}

}  // namespace mlpf
