// mlp_fused.cuh -- one training step of the surrogate network in two
// kernels, for networks whose layers fit a block's shared memory (inputs and
// hidden width <= 128, outputs <= 16, at most 8 layers).
//
// mlp_chunk_kernel: every block carries chunks of R = 32 batch rows through
// the forward pass, the loss and the backward pass.  All activations of a
// chunk stay in shared memory.  The weights are staged there one layer at a
// time from a bf16 copy kept in global memory in exactly the shared-memory
// layout (rows and columns padded with zeros); the copy for the next product
// is in flight (cp.async) while the current one runs, when two staging
// buffers fit.  The products are block-wide sums of warp tiles of mma.sync
// m16n8k16 (bf16 in, FP32 accumulation) with ldmatrix fragment loads; the
// backward products take the transposed fragments (ldmatrix .trans) of dz,
// of the layer inputs and of W, so nothing is transposed in memory.  The
// rounding points are those of the layer-by-layer
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
constexpr int NT = 512;        // threads per block (16 warps)
constexpr int NJ = 2;          // 8-column tiles per warp job of a block product
constexpr int MAXW = 128;      // largest input or hidden width
constexpr int MAXO = 16;       // largest output width
constexpr int MAXL = 8;        // most layers (hidden and output)

__host__ __device__ constexpr int kpad(int d) { return (d + 15) & ~15; }   // extent as a K dimension (16-steps)
__host__ __device__ constexpr int npad(int d) { return (d + 7) & ~7; }     // extent as an N dimension (8-tiles)
// row stride in bf16 elements of a K-contiguous operand: 8 elements past the
// K extent, so the 8 rows x 4 column pairs of a fragment load fall in 32
// distinct banks for every K extent that is a multiple of 16
__host__ __device__ constexpr int ldk(int d) { return kpad(d) + 8; }

// row stride in floats of the FP32 per-row arrays (z, dz): 4 past the width,
// so the 8 rows of an accumulator fragment start in different banks
__host__ __device__ constexpr int zld(int d) { return d + 4; }

// sizes, parameter offsets and the shared-memory layout (byte offsets)
struct Net {
    int nl, maxd;                           // layers; widest layer output
    int din[MAXL], dout[MAXL];
    long long woff[MAXL], boff[MAXL], qoff[MAXL];
    long long nparams;
    long long fo[MAXL];                     // element offset of the staged copy of W_l: [kpad(dout)][ldk(din)]
    long long nstaged;                      // elements in the staged copies
    int nbuf;                               // staging buffers (2: the next copy is prefetched)
    unsigned oH[MAXL];                      // bf16 [R][ldk(din[l])]: input of layer l
    unsigned oZ[MAXL];                      // float [R][zld(dout[l])]: pre-activation of hidden layer l
    unsigned oW[2];                         // bf16: staged weight matrices
    unsigned oB;                            // float [nl][maxd]: biases
    unsigned oD16[2];                       // bf16 [R][ldk(maxd)]: dz rounded, two buffers
    unsigned oD32;                          // float [R][zld(maxd)]: dz
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
    int maxd = 0;
    for (int l = 0; l < nl; ++l) {
        if (din[l] < 1 || din[l] > MAXW || dout[l] < 1) return false;
        if (l < nl - 1 ? dout[l] > MAXW : dout[l] > MAXO) return false;
        n.din[l] = din[l];
        n.dout[l] = dout[l];
        n.woff[l] = woff[l];
        n.boff[l] = boff[l];
        n.qoff[l] = qoff[l];
        maxd = dout[l] > maxd ? dout[l] : maxd;
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
        if (l < nl - 1) n.oZ[l] = take(sizeof(float) * R * zld(dout[l]));
        // W as [n][k] for the forward product and as [k][n] (transposed
        // fragments) for the backward one: rows to the next 16
        const size_t w = static_cast<size_t>(kpad(dout[l])) * ldk(din[l]);
        wsz = w > wsz ? w : wsz;
        n.fo[l] = st;
        st += static_cast<long long>(w);
    }
    n.nstaged = st;
    n.oB = take(sizeof(float) * nl * maxd);
    n.oW[0] = take(sizeof(bf16) * wsz);
    n.oD16[0] = take(sizeof(bf16) * R * ldk(maxd));
    n.oD16[1] = take(sizeof(bf16) * R * ldk(maxd));
    n.oD32 = take(sizeof(float) * R * zld(maxd));
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

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// four / two 8x8 bf16 matrices from shared memory, lane i naming row i % 8 of
// matrix i / 8; .trans hands out the transposed fragments
__device__ __forceinline__ void ldsm4(unsigned r[4], const bf16 *p, bool trans)
{
    if (trans)
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)) : "memory");
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)) : "memory");
}

__device__ __forceinline__ void ldsm2(unsigned r[2], const bf16 *p, bool trans)
{
    if (trans)
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(smem_u32(p)) : "memory");
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(smem_u32(p)) : "memory");
}

// Block-wide C = A B over shared-memory bf16 operands, with FP32 sums.
// AT = false: A stored [m][k] (row stride lda); AT = true: stored [k][m].
// BT = false: B stored [n][k] (row stride ldb); BT = true: stored [k][n].
// M = 16 Mt, N = 8 Nt, K = 16 Ks, every stored row 16-byte aligned and the
// operands zero past their extents up to those multiples.  Each warp takes a
// 16-row strip of up to NJ 8-column tiles at a time and hands the results
// to epi(row, col, v(row, col), v(row, col + 1)) for even col.  Jobs of NJ
// tiles keep every warp of the block busy on the smallest products.
template <bool AT, bool BT, typename Epi>
__device__ __forceinline__ void bgemm(const bf16 *A, int lda, const bf16 *B, int ldb, int Mt, int Nt, int Ks, Epi epi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3, rr = lane & 7, q = lane >> 3;
    const int Nq = (Nt + NJ - 1) / NJ;
    for (int job = warp; job < Mt * Nq; job += NT / 32) {
        const int mt = job / Nq, nq = job - (job / Nq) * Nq;
        float acc[NJ][4];
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
        for (int ks = 0; ks < Ks; ++ks) {
            const int k0 = 16 * ks, m0 = 16 * mt;
            unsigned a[4];
            // matrix q of the A fragment: rows m0 + 8 (q & 1), columns k0 + 8 (q >> 1)
            if (AT) ldsm4(a, A + (k0 + rr + 8 * (q >> 1)) * lda + m0 + 8 * (q & 1), true);
            else ldsm4(a, A + (m0 + rr + 8 * (q & 1)) * lda + k0 + 8 * (q >> 1), false);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int nt = NJ * nq + j;
                if (nt < Nt) {
                    // matrix q & 1 of the B fragment: k0 + 8 (q & 1)
                    unsigned b[2];
                    if (BT) ldsm2(b, B + (k0 + rr + 8 * (q & 1)) * ldb + 8 * nt, true);
                    else ldsm2(b, B + (8 * nt + rr) * ldb + k0 + 8 * (q & 1), false);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
                        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
                }
            }
        }
        // acc[j][0, 1]: row g, columns 2 t, 2 t + 1 of tile NJ nq + j; acc[j][2, 3]: row g + 8
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int nt = NJ * nq + j;
            if (nt < Nt) {
                epi(16 * mt + g, 8 * nt + 2 * t, acc[j][0], acc[j][1]);
                epi(16 * mt + g + 8, 8 * nt + 2 * t, acc[j][2], acc[j][3]);
            }
        }
    }
}

// Staging step s of a chunk: W of layer s (forward, s < nl) or of layer
// 2 nl - 1 - s (backward), as 16-byte cp.async into Ws, one commit group.
__device__ __forceinline__ void stage_async(const Net &net, int s, bf16 *Ws, const bf16 *__restrict__ WS)
{
    const int l = s < net.nl ? s : 2 * net.nl - 1 - s;
    const int n = kpad(net.dout[l]) * ldk(net.din[l]);
    const unsigned dst = smem_u32(Ws);
    const bf16 *src = WS + net.fo[l];
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
// [gridDim.x] receive its sums over its chunks.  step (graph replay, or
// null): the step index, advanced here by one (it starts a call at -1), so
// that the reduction kernel of the same step reads it.
template <bool TRAIN>
__global__ void __launch_bounds__(NT) mlp_chunk_kernel(Net net, const float *__restrict__ P, const bf16 *__restrict__ WS,
                                                       const float *__restrict__ X, const float *__restrict__ T, int B,
                                                       float *__restrict__ Y, float *__restrict__ part,
                                                       float *__restrict__ lpart, int *step)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (step && blockIdx.x == 0 && tid == 0) *step += 1;
    const int nl = net.nl, n_in = net.din[0], maxd = net.maxd, LDD = ldk(maxd), ZD = zld(maxd);
    float *D32 = reinterpret_cast<float *>(sm + net.oD32);
    const long long NP = net.nparams;
    const float sc = 2.0f / static_cast<float>(static_cast<long long>(B) * net.dout[nl - 1]);
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
            // outside; a warp per row, the row's loads issued together
            bf16 *H0 = reinterpret_cast<bf16 *>(sm + net.oH[0]);
            const int kp = kpad(n_in), ls = ldk(n_in);
            for (int r = warp; r < R; r += NT / 32) {
                float x[MAXW / 32];
#pragma unroll
                for (int u = 0; u < MAXW / 32; ++u) {
                    const int k = lane + 32 * u;
                    x[u] = (r < nr && k < n_in) ? X[static_cast<long long>(r0 + r) * n_in + k] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < MAXW / 32; ++u) {
                    const int k = lane + 32 * u;
                    if (k < kp) H0[r * ls + k] = __float2bfloat16_rn(x[u]);
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
                const int ln = ldk(dn), zs = zld(dn);
                bgemm<false, false>(Hl, ldk(di), Ws, ldk(di), R / 16, npad(dn) / 8, kpad(di) / 16,
                                    [&](int r, int c, float v0, float v1) {
                                        if (c < dn) {
                                            const float z = v0 + bias[c];
                                            Z[r * zs + c] = z;
                                            Hn[r * ln + c] = __float2bfloat16_rn(gelu(z));
                                        }
                                        if (c + 1 < dn) {
                                            const float z = v1 + bias[c + 1];
                                            Z[r * zs + c + 1] = z;
                                            Hn[r * ln + c + 1] = __float2bfloat16_rn(gelu(z));
                                        }
                                    });
            } else {
                bgemm<false, false>(Hl, ldk(di), Ws, ldk(di), R / 16, npad(dn) / 8, kpad(di) / 16,
                                    [&](int r, int c0, float v0, float v1) {
                                        for (int e = 0; e < 2; ++e) {
                                            const int c = c0 + e;
                                            if (c >= dn) break;
                                            const float y = (e ? v1 : v0) + bias[c];
                                            if (!TRAIN) {
                                                if (r < nr) Y[static_cast<long long>(r0 + r) * dn + c] = y;
                                                continue;
                                            }
                                            // d loss / d y of the mean squared error; rows past B add nothing
                                            const float d =
                                                (r < nr) ? y - T[static_cast<long long>(r0 + r) * dn + c] : 0.f;
                                            lacc += d * d;
                                            D32[r * ZD + c] = sc * d;
                                            D16[r * LDD + c] = __float2bfloat16_rn(sc * d);
                                        }
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
                for (int r = 0; r < R; ++r) s += D32[r * ZD + c];
                pb[c] = first ? s : pb[c] + s;
            }
            const bf16 *Ws = nullptr;
            if (l > 0) {
                zero_cols(reinterpret_cast<bf16 *>(sm + net.oD16[(l - 1) & 1]), LDD, di, kpad(di));
                Ws = staged(2 * nl - 1 - l, ch);
            }
            __syncthreads();
            // dW_l += dz_l^T H_l over the chunk's rows: both operands stored
            // with the rows of the chunk as K
            float *pw = part + static_cast<long long>(blockIdx.x) * NP + net.woff[l];
            bgemm<true, true>(D16, LDD, Hl, ldk(di), kpad(dn) / 16, npad(di) / 8, R / 16,
                              [&](int r, int c, float v0, float v1) {
                                  if (r >= dn) return;
                                  float *q = pw + static_cast<long long>(r) * di + c;
                                  if (c < di) q[0] = first ? v0 : q[0] + v0;
                                  if (c + 1 < di) q[1] = first ? v1 : q[1] + v1;
                              });
            if (l > 0) {
                // dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1}), W_l stored [k = out][n = in]
                const float *Zp = reinterpret_cast<const float *>(sm + net.oZ[l - 1]);
                bf16 *Dn = reinterpret_cast<bf16 *>(sm + net.oD16[(l - 1) & 1]);
                const int zs = zld(di);
                bgemm<false, true>(D16, LDD, Ws, ldk(di), R / 16, npad(di) / 8, kpad(dn) / 16,
                                   [&](int r, int c, float v0, float v1) {
                                       if (c < di) {
                                           const float dz = v0 * gelu_grad(Zp[r * zs + c]);
                                           D32[r * ZD + c] = dz;
                                           Dn[r * LDD + c] = __float2bfloat16_rn(dz);
                                       }
                                       if (c + 1 < di) {
                                           const float dz = v1 * gelu_grad(Zp[r * zs + c + 1]);
                                           D32[r * ZD + c + 1] = dz;
                                           Dn[r * LDD + c + 1] = __float2bfloat16_rn(dz);
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
        if (lane == 0) red[warp] = lacc;
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
    float *hist;           // if set (with bc): the loss also goes to hist[*cnt]
};

// weight i (a parameter index) rounded to bf16 into the staged copy WS
// (W_l at [k][n] with padded rows) and, if wq is set, the row-major copy
__device__ __forceinline__ void put_weight(const Net &net, long long i, float w, bf16 *WS, bf16 *wq)
{
    for (int l = 0; l < net.nl; ++l) {
        if (i < net.woff[l] || i >= net.boff[l]) continue;
        const bf16 b = __float2bfloat16_rn(w);
        const long long j = i - net.woff[l];
        const int di = net.din[l], k = static_cast<int>(j / di), n = static_cast<int>(j - (j / di) * di);
        WS[net.fo[l] + static_cast<long long>(k) * ldk(di) + n] = b;
        if (wq) wq[net.qoff[l] + j] = b;
    }
}

// the staged copy of every weight from the FP32 parameters (its padding
// stays as cleared at creation)
__global__ void mlp_stage_copies_kernel(Net net, const float *__restrict__ p, bf16 *WS)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < net.nparams;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        put_weight(net, i, p[i], WS, nullptr);
}

constexpr int RP = 64;          // parameters per block of the reduction
constexpr int RQ = 4;           // partial sums per parameter (RP x RQ threads)

// Sum of the G slices of every parameter's gradient (quarter q of the
// slices by threads q, then the four quarters in order: a fixed order), and
// of the G loss sums.  ADAM = false: grad and loss out.  ADAM = true: loss
// out, Adam step on p with moments m, v, and the bf16 copies of every
// weight.  Blocks of RP x RQ threads, RP parameters each.
template <bool ADAM>
__global__ void __launch_bounds__(RP * RQ)
mlp_reduce_kernel(Net net, int G, const float *__restrict__ part, const float *__restrict__ lpart, long long nsum,
                  float *__restrict__ grad, float *__restrict__ loss, float *p, float *m, float *v, bf16 *WS,
                  bf16 *wq, Adam o)
{
    __shared__ float red[RQ][RP];
    const long long NP = net.nparams;
    const int j = threadIdx.x % RP, qr = threadIdx.x / RP;
    const long long i = static_cast<long long>(blockIdx.x) * RP + j;
    const int qg = (G + RQ - 1) / RQ, c0 = qr * qg, c1 = min(G, c0 + qg);
    float gq = 0.f;
    if (i < NP) {
#pragma unroll 8
        for (int c = c0; c < c1; ++c) gq += part[static_cast<long long>(c) * NP + i];
    }
    red[qr][j] = gq;
    __syncthreads();
    if (qr == 0 && i < NP) {
        const float gi = (red[0][j] + red[1][j]) + (red[2][j] + red[3][j]);
        if (!ADAM) {
            grad[i] = gi;
        } else {
            float bc1 = o.bc1, bc2 = o.bc2;
            if (o.bc) {
                const int k = *o.cnt;
                bc1 = o.bc[2 * k];
                bc2 = o.bc[2 * k + 1];
            }
            const float mi = o.b1 * m[i] + (1.0f - o.b1) * gi;
            const float vi = o.b2 * v[i] + (1.0f - o.b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            const float pi = p[i] - o.lr * (mi / bc1) / (sqrtf(vi / bc2) + o.eps);
            p[i] = pi;
            put_weight(net, i, pi, WS, wq);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int c = 0; c < G; ++c) s += lpart[c];
        *loss = s / static_cast<float>(nsum);
        if (ADAM && o.bc && o.hist) o.hist[*o.cnt] = s / static_cast<float>(nsum);
    }
}

}  // namespace mlpf
