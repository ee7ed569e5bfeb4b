// Surrogate MLP: lattice parameters -> final emittances, trained with a
// Sobolev loss on the values and the exact dual-number derivatives the PIC
// produces. The network is n_in -> width (x hidden, GELU) -> n_out. Forward
// mode carries, for every sample, one primal row and n_in tangent rows (the
// derivatives of every activation with respect to the inputs), so a batch of
// B samples is a GEMM over R = B (n_in + 1) rows; the tangent rows share the
// weights, skip the bias, and pass the nonlinearity as GELU'(h) times their
// pre-activation. The backward pass runs reverse mode through both paths
// (the tangent path depends on h through GELU', hence GELU'').
//
// GEMMs: BF16 operands, FP32 accumulation, tensor cores through
// mma.sync.m16n8k16 (row.col), 64 x 64 block tiles staged through shared
// memory with bounds-checked loads (any M, N, K; any operand strides, so the
// transposed products of the backward pass need no transposed copies).
// Weights live in FP32 (Adam) with BF16 copies for the GEMMs; activations
// are stored in BF16.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ad_pic.h"

namespace {

// ------------------------------------------------------------------ GEMM

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;

// One operand tile [rows][BK] of X(r, k) = X[r * sr + k * sk] (BF16) on its
// way to shared memory, in two steps so the next tile's loads can be in flight
// while the current one is multiplied: tile_load reads it into registers
// (16-byte vectors along k, k contiguous, or along r, r contiguous: the
// transposed operands of the backward pass, where the strides and the tile
// allow), tile_store writes them to shared memory. Tiles that allow neither
// (ragged edges, odd strides) are read with bounds-checked scalar loads in
// tile_store itself. 128 threads: two vectors each.
constexpr int kGemmThreads = 128;
struct TileRegs {
    uint4 v[BM * BK / 8 / kGemmThreads];
    int mode;                 // 1 along k, 2 along r, 0 scalar in tile_store
};
__device__ __forceinline__ void tile_load(TileRegs& t, const __nv_bfloat16* __restrict__ X, int64_t sr, int64_t sk,
                                          int r0, int R, int k0, int K, bool vk, bool vr) {
    t.mode = (vk && k0 + BK <= K) ? 1 : ((vr && r0 + BM <= R) ? 2 : 0);
#pragma unroll
    for (int i = 0; i < BM * BK / 8 / kGemmThreads; ++i) {
        const int q = threadIdx.x + i * kGemmThreads;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t.mode == 1) {
            const int r = q / (BK / 8), c = (q % (BK / 8)) * 8, gr = r0 + r;
            if (gr < R) v = *reinterpret_cast<const uint4*>(X + gr * sr + (k0 + c));
        } else if (t.mode == 2) {
            const int c = q / (BM / 8), r = (q % (BM / 8)) * 8, gk = k0 + c;
            if (gk < K) v = *reinterpret_cast<const uint4*>(X + (r0 + r) + gk * sk);
        }
        t.v[i] = v;
    }
}
__device__ __forceinline__ void tile_store(const TileRegs& t, __nv_bfloat16 (*Xs)[BK + PADK],
                                           const __nv_bfloat16* __restrict__ X, int64_t sr, int64_t sk, int r0, int R,
                                           int k0, int K) {
    if (t.mode == 1) {
#pragma unroll
        for (int i = 0; i < BM * BK / 8 / kGemmThreads; ++i) {
            const int q = threadIdx.x + i * kGemmThreads;
            const int r = q / (BK / 8), c = (q % (BK / 8)) * 8;
            *reinterpret_cast<uint4*>(&Xs[r][c]) = t.v[i];
        }
    } else if (t.mode == 2) {
#pragma unroll
        for (int i = 0; i < BM * BK / 8 / kGemmThreads; ++i) {
            const int q = threadIdx.x + i * kGemmThreads;
            const int c = q / (BM / 8), r = (q % (BM / 8)) * 8;
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&t.v[i]);
#pragma unroll
            for (int j = 0; j < 8; ++j) Xs[r + j][c] = e[j];
        }
    } else {
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        for (int q = threadIdx.x; q < BM * BK; q += kGemmThreads) {
            const int r = sk == 1 ? q / BK : q % BM, c = sk == 1 ? q % BK : q / BM;
            const int gr = r0 + r, gk = k0 + c;
            Xs[r][c] = (gr < R && gk < K) ? X[gr * sr + gk * sk] : zero;
        }
    }
}

__device__ __forceinline__ float phi(float x) { return 0.3989422804014327f * __expf(-0.5f * x * x); }
__device__ __forceinline__ float Phi(float x) { return 0.5f * (1.f + erff(x * 0.7071067811865476f)); }

// What the GEMM does with its 64 x 64 tile after the products, on the rows
// r = s S + c of the Sobolev network (c = 0 primal, c > 0 the tangent of input
// c - 1; a tile holds whole samples, 64 % S == 0). EPI_STORE stores C. The
// others store C and also do, on the tile:
//   EPI_HIDDEN  (forward, hidden layer) primal rows h += b, a = GELU(h) =
//               h Phi(h); tangent rows a = GELU'(h_primal) h (no bias);
//               a goes to act (BF16 rows of the next layer's input);
//   EPI_OUTPUT  (forward, output layer) primal rows += b;
//   EPI_BACKWARD (backward into a hidden layer's pre-activations, from dL/da
//               of that layer's output; Hp its pre-activations) per sample and
//               unit: dL/dh = G_p GELU'(h) + sum_c G_c t_c GELU''(h), the
//               tangent rows G_c GELU'(h); FP32 in C, BF16 copy in act.
enum { EPI_STORE = 0, EPI_HIDDEN, EPI_OUTPUT, EPI_BACKWARD };
struct Epi {
    int S;
    const float* bias;
    __nv_bfloat16* act;
    const float* Hp;
};

// C[m][n] (ldc) = sum_k A(m, k) B(n, k) + beta * C[m][n], with
// A(m, k) = A[m * sam + k * sak] and B(n, k) = B[n * sbn + k * sbk] (BF16).
// blockIdx.z splits K: with split > 1 each slice writes its partial sum to
// C + z * M * N (row-major [M][N], beta ignored) for split_reduce_kernel.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 4) gemm_bf16_kernel(int M, int N, int K, int kslice, const __nv_bfloat16* __restrict__ A,
                                                        int64_t sam, int64_t sak, const __nv_bfloat16* __restrict__ B,
                                                        int64_t sbn, int64_t sbk, float* __restrict__ C, int64_t ldc,
                                                        float beta, bool avk, bool avr, bool bvk, bool bvr, Epi ep) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PADK];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    if (gridDim.z > 1) {
        C += (int64_t)blockIdx.z * M * N;
        ldc = N;
        beta = 0.f;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;     // 2 x 2 warps of 32 x 32
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    TileRegs ra, rb;
    tile_load(ra, A, sam, sak, m0, M, kb, ke, avk, avr);
    tile_load(rb, B, sbn, sbk, n0, N, kb, ke, bvk, bvr);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        tile_store(ra, As, A, sam, sak, m0, M, k0, ke);
        tile_store(rb, Bs, B, sbn, sbk, n0, N, k0, ke);
        __syncthreads();
        if (k0 + BK < ke) {                  // the next tile's loads overlap this tile's products
            tile_load(ra, A, sam, sak, m0, M, k0 + BK, ke, avk, avr);
            tile_load(rb, B, sbn, sbk, n0, N, k0 + BK, ke, bvk, bvr);
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + grp;
                a[i][0] = *reinterpret_cast<const unsigned*>(&As[r][kk + tig * 2]);
                a[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + tig * 2]);
                a[i][2] = *reinterpret_cast<const unsigned*>(&As[r][kk + tig * 2 + 8]);
                a[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + tig * 2 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + grp;
                b[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + tig * 2]);
                b[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + tig * 2 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
        }
        __syncthreads();
    }
    if constexpr (EPI == EPI_STORE) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = m0 + wm + i * 16 + grp + (q >= 2 ? 8 : 0);
                    const int c = n0 + wn + j * 8 + tig * 2 + (q & 1);
                    if (r < M && c < N) {
                        float* p = C + (int64_t)r * ldc + c;
                        *p = acc[i][j][q] + (beta != 0.f ? beta * *p : 0.f);
                    }
                }
    } else {
        // the tile through shared memory, so each sample's rows meet
        __shared__ float Cs[BM][BN + 1];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Cs[wm + i * 16 + grp + (q >= 2 ? 8 : 0)][wn + j * 8 + tig * 2 + (q & 1)] = acc[i][j][q];
        __syncthreads();
        const int S = ep.S;
        if constexpr (EPI == EPI_HIDDEN || EPI == EPI_OUTPUT) {
            for (int t = threadIdx.x; t < BM * BN; t += blockDim.x) {
                const int rl = t / BN, cl = t % BN;
                const int r = m0 + rl, c = n0 + cl;
                if (r >= M || c >= N) continue;
                const int cs = rl % S;
                const float v = Cs[rl][cl];
                const int64_t at = (int64_t)r * ldc + c;
                if (EPI == EPI_OUTPUT) {
                    C[at] = cs == 0 ? v + ep.bias[c] : v;
                } else if (cs == 0) {
                    const float hh = v + ep.bias[c];
                    C[at] = hh;
                    ep.act[(int64_t)r * N + c] = __float2bfloat16(hh * Phi(hh));
                } else {
                    const float hp = Cs[rl - cs][cl] + ep.bias[c];
                    const float d1 = Phi(hp) + hp * phi(hp);
                    C[at] = v;
                    ep.act[(int64_t)r * N + c] = __float2bfloat16(d1 * v);
                }
            }
        } else {
            for (int t = threadIdx.x; t < (BM / S) * BN; t += blockDim.x) {
                const int sl = t / BN, cl = t % BN;
                const int rp = m0 + sl * S, c = n0 + cl;
                if (rp >= M || c >= N) continue;
                const int64_t p = (int64_t)rp * ldc + c;
                const float hh = ep.Hp[p];
                const float d1 = Phi(hh) + hh * phi(hh);
                const float d2 = phi(hh) * (2.f - hh * hh);
                float gh = Cs[sl * S][cl] * d1;
                for (int cc = 1; cc < S; ++cc) {
                    const int64_t q = p + (int64_t)cc * ldc;
                    const float g = Cs[sl * S + cc][cl];
                    gh += g * ep.Hp[q] * d2;
                    const float gt = g * d1;
                    C[q] = gt;
                    ep.act[q] = __float2bfloat16(gt);
                }
                C[p] = gh;
                ep.act[p] = __float2bfloat16(gh);
            }
        }
    }
}

// C[m][n] = sum over the split slices of the partials, in slice order
__global__ void split_reduce_kernel(const float* __restrict__ part, int split, int M, int N, float* __restrict__ C,
                                    int64_t ldc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * N) return;
    float s = 0.f;
    for (int z = 0; z < split; ++z) s += part[(int64_t)z * M * N + t];
    C[(t / N) * ldc + t % N] = s;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// K slices of a GEMM whose tiles alone do not fill the GPU (the weight
// gradients: a few 64 x 64 tiles, K = the batch's rows): enough slices for
// about two tiles per SM, each at least 8 k-steps long, within the workspace
constexpr int kMaxSplit = 32;
int split_of(int M, int N, int K) {
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int split = 1;
    while (split < kMaxSplit && tiles * split < 304 && K / (split * 2) >= 8 * BK) split *= 2;
    return split;
}

void gemm(int M, int N, int K, const __nv_bfloat16* A, int64_t sam, int64_t sak, const __nv_bfloat16* B, int64_t sbn,
          int64_t sbk, float* C, int64_t ldc, float beta, cudaStream_t s, float* ws = nullptr, int epi = EPI_STORE,
          Epi ep = Epi{1, nullptr, nullptr, nullptr}) {
    const bool avk = sak == 1 && sam % 8 == 0 && aligned16(A), avr = sam == 1 && sak % 8 == 0 && aligned16(A);
    const bool bvk = sbk == 1 && sbn % 8 == 0 && aligned16(B), bvr = sbn == 1 && sbk % 8 == 0 && aligned16(B);
    const int split = (ws && beta == 0.f && epi == EPI_STORE) ? split_of(M, N, K) : 1;
    const int kslice = ((K + split * BK - 1) / (split * BK)) * BK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, split);
    float* out = split > 1 ? ws : C;
#define ADPIC_GEMM(E) gemm_bf16_kernel<E><<<grid, kGemmThreads, 0, s>>>(M, N, K, kslice, A, sam, sak, B, sbn, sbk, out, ldc, \
                                                                 beta, avk, avr, bvk, bvr, ep)
    switch (epi) {
        case EPI_HIDDEN: ADPIC_GEMM(EPI_HIDDEN); break;
        case EPI_OUTPUT: ADPIC_GEMM(EPI_OUTPUT); break;
        case EPI_BACKWARD: ADPIC_GEMM(EPI_BACKWARD); break;
        default: ADPIC_GEMM(EPI_STORE); break;
    }
#undef ADPIC_GEMM
    if (split > 1)
        split_reduce_kernel<<<(unsigned)(((int64_t)M * N + 255) / 256), 256, 0, s>>>(ws, split, M, N, C, ldc);
}

// ------------------------------------------------------------------ elementwise


// rows r = s * S + c (S = n_in + 1; c = 0 primal, c > 0 tangent of input c-1).
// Primal rows of a hidden layer: h += b, a = GELU(h) (tangent rows follow in
// act_fwd_tangent_kernel, once every primal h has its bias). H keeps the
// pre-activations (FP32) for the backward pass.
__global__ void act_fwd_kernel(float* __restrict__ H, const float* __restrict__ b, __nv_bfloat16* __restrict__ Aout,
                               int R, int S, int width) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * width) return;
    const int r = (int)(t / width), j = (int)(t % width);
    if (r % S != 0) return;
    const float h = H[t] + b[j];
    H[t] = h;
    Aout[t] = __float2bfloat16(h * Phi(h));
}

// tangent rows in a second pass, after every primal h has its bias
__global__ void act_fwd_tangent_kernel(const float* __restrict__ H, __nv_bfloat16* __restrict__ Aout, int R, int S,
                                       int width) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * width) return;
    const int r = (int)(t / width), j = (int)(t % width);
    const int c = r % S;
    if (c == 0) return;
    const float hp = H[(int64_t)(r - c) * width + j];
    const float d1 = Phi(hp) + hp * phi(hp);
    Aout[t] = __float2bfloat16(d1 * H[t]);
}

// Sobolev loss of the output rows Y [R][n_out] (bias already added on primal
// rows) against targets t [B][n_out] and dt [B][n_out][n_in]; writes the
// gradient dY (FP32 and BF16) and accumulates the loss (FP64 atomics).
__global__ void sobolev_kernel(const float* __restrict__ Y, const float* __restrict__ tgt, const float* __restrict__ dtgt,
                               int B, int S, int n_in, int n_out, float lam, float* __restrict__ dY,
                               __nv_bfloat16* __restrict__ dYb, double* __restrict__ loss) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int R = B * S;
    double l = 0.0;
    if (t < (int64_t)R * n_out) {
        const int r = (int)(t / n_out), o = (int)(t % n_out);
        const int s = r / S, c = r % S;
        float g;
        if (c == 0) {
            const float e = Y[t] - tgt[s * n_out + o];
            l = (double)e * e;
            g = 2.f * e / (float)B;
        } else {
            const float e = Y[t] - dtgt[((int64_t)s * n_out + o) * n_in + (c - 1)];
            l = (double)lam * e * e;
            g = 2.f * lam * e / (float)B;
        }
        dY[t] = g;
        dYb[t] = __float2bfloat16(g);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l / (double)B);
}

// backward through a hidden layer: G [R][width] holds dL/da (primal rows) and
// dL/d(tangent a) (tangent rows) on entry; on exit dL/dh and dL/d(tangent h)
// (FP32 in G, BF16 copy in Gb). H holds the pre-activations.
__global__ void act_bwd_kernel(float* __restrict__ G, const float* __restrict__ H, __nv_bfloat16* __restrict__ Gb, int R,
                               int S, int width) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // one thread per (sample, unit)
    const int B = R / S;
    if (t >= (int64_t)B * width) return;
    const int s = (int)(t / width), j = (int)(t % width);
    const int64_t p = (int64_t)s * S * width + j;
    const float h = H[p];
    const float d1 = Phi(h) + h * phi(h);
    const float d2 = phi(h) * (2.f - h * h);
    float gh = G[p] * d1;
    for (int c = 1; c < S; ++c) {
        const int64_t q = p + (int64_t)c * width;
        gh += G[q] * H[q] * d2;
        const float gt = G[q] * d1;
        G[q] = gt;
        Gb[q] = __float2bfloat16(gt);
    }
    G[p] = gh;
    Gb[p] = __float2bfloat16(gh);
}

// db[j] = sum over primal rows of G[r][j]: a block per 32 columns, its 8
// warps over interleaved samples, then the 8 partial sums in order
__global__ void bias_grad_kernel(const float* __restrict__ G, int B, int S, int width, float* __restrict__ db) {
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (j < width)
        for (int b = w; b < B; b += 8) s += G[(int64_t)b * S * width + j];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < width) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][lane];
        db[j] = t;
    }
}

__global__ void add_bias_primal_kernel(float* __restrict__ Y, const float* __restrict__ b, int R, int S, int n_out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * n_out) return;
    const int r = (int)(t / n_out);
    if (r % S == 0) Y[t] += b[t % n_out];
}

// inputs: primal rows x (BF16), tangent row c carries the unit vector e_{c-1}
__global__ void input_rows_kernel(const float* __restrict__ x, int B, int S, int n_in, __nv_bfloat16* __restrict__ A0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * S * n_in) return;
    const int r = (int)(t / n_in), k = (int)(t % n_in);
    const int s = r / S, c = r % S;
    A0[t] = __float2bfloat16(c == 0 ? x[(int64_t)s * n_in + k] : (c - 1 == k ? 1.f : 0.f));
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[t] -= upd;
    pb[t] = __float2bfloat16(p[t]);
}

// Adam with the step counter on the device (graph-replayable): lr follows the
// geometric schedule lr0 (lr1 / lr0)^(s / total) of the step s of the run;
// thread 0 of the last block advances the counters after every thread has
// read them (a grid-wide count of finished blocks)
__global__ void adam_dev_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n, float lr0, float lr1,
                                int total, float b1, float b2, float eps, int64_t* __restrict__ ctr,
                                unsigned* __restrict__ done) {
    const int64_t step = ctr[0] + 1;               // Adam's step count (1-based)
    const float frac = total > 1 ? (float)ctr[1] / (float)(total - 1) : 0.f;
    const float lr = lr0 * powf(lr1 / lr0, frac);
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) {
        const float gg = g[t];
        const float mm = b1 * m[t] + (1.f - b1) * gg;
        const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
        m[t] = mm;
        v[t] = vv;
        p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        pb[t] = __float2bfloat16(p[t]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            ctr[0] += 1;
            ctr[1] += 1;
            ctr[2] += 1;
            *done = 0u;
            __threadfence();
        }
    }
}

// the mini-batch of the current step: B samples from the device-resident
// training set, taken in the (shuffled-at-upload) order, wrapping around
__global__ void gather_batch_kernel(const float* __restrict__ X, const float* __restrict__ T,
                                    const float* __restrict__ DT, int n, int B, int n_in, int n_out,
                                    const int64_t* __restrict__ ctr, float* __restrict__ x, float* __restrict__ t,
                                    float* __restrict__ dt) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int per = n_in + n_out + n_out * n_in;
    if (k >= (int64_t)B * per) return;
    const int r = (int)(k / per), c = (int)(k % per);
    const int64_t src = (ctr[2] * (int64_t)B + r) % n;
    if (c < n_in) x[(int64_t)r * n_in + c] = X[src * n_in + c];
    else if (c < n_in + n_out) t[(int64_t)r * n_out + (c - n_in)] = T[src * n_out + (c - n_in)];
    else dt[(int64_t)r * n_out * n_in + (c - n_in - n_out)] = DT[src * n_out * n_in + (c - n_in - n_out)];
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = __float2bfloat16(a[t]);
}

unsigned nb(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

struct ad_pic_mlp {
    int n_in = 0, width = 0, hidden = 0, n_out = 0, max_batch = 0, S = 0;
    int layers = 0;                          // hidden + 1 dense layers
    std::vector<int> in_dim, out_dim;
    std::vector<int64_t> w_off, b_off;       // offsets in the flat parameter vector
    int64_t n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 parameters, gradient, Adam moments
    __nv_bfloat16* pb = nullptr;            // BF16 copy of the parameters
    std::vector<float*> H;                   // per layer pre-activations [R][out] (FP32)
    std::vector<__nv_bfloat16*> A;           // per layer inputs [R][in] (BF16); A[0] = input rows
    float* G = nullptr;                      // gradient rows [R][max width] (FP32)
    float* G2 = nullptr;
    float* ws = nullptr;                     // split-K partial sums of the weight gradients
    __nv_bfloat16* Gb = nullptr;
    float *x = nullptr, *t = nullptr, *dt = nullptr;
    double* loss = nullptr;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    // device-resident training set and the counters of ad_pic_mlp_train
    float *dx = nullptr, *dtg = nullptr, *ddt = nullptr;
    int n_data = 0, data_cap = 0;
    int64_t* ctr = nullptr;                  // [0] Adam steps, [1] step in the current run, [2] batches drawn
    unsigned* done = nullptr;
    cudaGraphExec_t train_graph = nullptr;
    int g_B = 0, g_total = 0;
    float g_lam = 0.f, g_lr0 = 0.f, g_lr1 = 0.f;
};

namespace {

int mlp_alloc(ad_pic_mlp* h, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return AD_PIC_ERR_OOM;
    }
    h->allocs.push_back(*p);
    return AD_PIC_OK;
}

// forward of a batch already uploaded in h->x; leaves H (pre-activations) and A (inputs)
void forward_rows(ad_pic_mlp* h, int B) {
    const int S = h->S, R = B * S;
    cudaStream_t s = h->stream;
    input_rows_kernel<<<nb((int64_t)R * h->n_in), 256, 0, s>>>(h->x, B, S, h->n_in, h->A[0]);
    for (int l = 0; l < h->layers; ++l) {
        const int in = h->in_dim[l], out = h->out_dim[l];
        const __nv_bfloat16* W = h->pb + h->w_off[l];          // [out][in]
        const bool hidden = l < h->layers - 1;
        if (BM % S == 0) {
            // activations in the GEMM's epilogue
            gemm(R, out, in, h->A[l], in, 1, W, in, 1, h->H[l], out, 0.f, s, nullptr,
                 hidden ? EPI_HIDDEN : EPI_OUTPUT, Epi{S, h->p + h->b_off[l], hidden ? h->A[l + 1] : nullptr, nullptr});
            continue;
        }
        gemm(R, out, in, h->A[l], in, 1, W, in, 1, h->H[l], out, 0.f, s);
        if (hidden) {
            act_fwd_kernel<<<nb((int64_t)R * out), 256, 0, s>>>(h->H[l], h->p + h->b_off[l], h->A[l + 1], R, S, out);
            act_fwd_tangent_kernel<<<nb((int64_t)R * out), 256, 0, s>>>(h->H[l], h->A[l + 1], R, S, out);
        } else {
            add_bias_primal_kernel<<<nb((int64_t)R * out), 256, 0, s>>>(h->H[l], h->p + h->b_off[l], R, S, out);
        }
    }
}

// loss and full gradient into h->g (needs h->x, h->t, h->dt uploaded)
void loss_grad(ad_pic_mlp* h, int B, float lam) {
    const int S = h->S, R = B * S;
    cudaStream_t s = h->stream;
    forward_rows(h, B);
    cudaMemsetAsync(h->loss, 0, sizeof(double), s);
    const int L = h->layers;
    sobolev_kernel<<<nb((int64_t)R * h->n_out), 256, 0, s>>>(h->H[L - 1], h->t, h->dt, B, S, h->n_in, h->n_out, lam,
                                                              h->G, h->Gb, h->loss);
    float* G = h->G;
    float* Gn = h->G2;
    for (int l = L - 1; l >= 0; --l) {
        const int in = h->in_dim[l], out = h->out_dim[l];
        // dW[o][i] = sum_r G[r][o] A[r][i]   (GEMM over the rows, both operands transposed in place)
        gemm(out, in, R, h->Gb, 1, out, h->A[l], 1, in, h->g + h->w_off[l], in, 0.f, s, h->ws);
        bias_grad_kernel<<<(unsigned)((out + 31) / 32), 256, 0, s>>>(G, B, S, out, h->g + h->b_off[l]);
        if (l == 0) break;
        // dA[r][i] = sum_o G[r][o] W[o][i]
        const __nv_bfloat16* W = h->pb + h->w_off[l];
        if (BM % S == 0) {
            gemm(R, in, out, h->Gb, out, 1, W, 1, in, Gn, in, 0.f, s, nullptr, EPI_BACKWARD,
                 Epi{S, nullptr, h->Gb, h->H[l - 1]});
        } else {
            gemm(R, in, out, h->Gb, out, 1, W, 1, in, Gn, in, 0.f, s);
            act_bwd_kernel<<<nb((int64_t)B * in), 256, 0, s>>>(Gn, h->H[l - 1], h->Gb, R, S, in);
        }
        float* tmp = G;
        G = Gn;
        Gn = tmp;
    }
}

int upload(ad_pic_mlp* h, const float* x, const float* t, const float* dt, int B) {
    cudaStream_t s = h->stream;
    if (x && cudaMemcpyAsync(h->x, x, sizeof(float) * B * h->n_in, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    if (t && cudaMemcpyAsync(h->t, t, sizeof(float) * B * h->n_out, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    if (dt && cudaMemcpyAsync(h->dt, dt, sizeof(float) * B * h->n_out * h->n_in, cudaMemcpyHostToDevice, s) !=
                  cudaSuccess)
        return AD_PIC_ERR_CUDA;
    return AD_PIC_OK;
}

}  // namespace

extern "C" {

int ad_pic_mlp_create(int n_in, int width, int hidden, int n_out, int max_batch, ad_pic_mlp** out) {
    if (!out) return AD_PIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || width < 1 || width > 4096 || hidden < 1 || hidden > 16 || n_out < 1 || n_out > 64 ||
        max_batch < 1 || (int64_t)max_batch * (n_in + 1) > (1 << 24))
        return AD_PIC_ERR_INVALID_ARG;
    ad_pic_mlp* h = new (std::nothrow) ad_pic_mlp();
    if (!h) return AD_PIC_ERR_OOM;
    h->n_in = n_in;
    h->width = width;
    h->hidden = hidden;
    h->n_out = n_out;
    h->max_batch = max_batch;
    h->S = n_in + 1;
    h->layers = hidden + 1;
    for (int l = 0; l < h->layers; ++l) {
        const int in = l == 0 ? n_in : width, o = l == h->layers - 1 ? n_out : width;
        h->in_dim.push_back(in);
        h->out_dim.push_back(o);
        h->w_off.push_back(h->n_params);
        h->n_params += (int64_t)in * o;
        h->b_off.push_back(h->n_params);
        h->n_params += o;
    }
    const int64_t R = (int64_t)max_batch * h->S;
    int st = 0;
    cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    st |= mlp_alloc(h, (void**)&h->p, sizeof(float) * h->n_params);
    st |= mlp_alloc(h, (void**)&h->g, sizeof(float) * h->n_params);
    st |= mlp_alloc(h, (void**)&h->m, sizeof(float) * h->n_params);
    st |= mlp_alloc(h, (void**)&h->v, sizeof(float) * h->n_params);
    st |= mlp_alloc(h, (void**)&h->pb, sizeof(__nv_bfloat16) * h->n_params);
    h->H.assign(h->layers, nullptr);
    h->A.assign(h->layers + 1, nullptr);
    for (int l = 0; l < h->layers; ++l) {
        st |= mlp_alloc(h, (void**)&h->H[l], sizeof(float) * R * h->out_dim[l]);
        st |= mlp_alloc(h, (void**)&h->A[l], sizeof(__nv_bfloat16) * R * h->in_dim[l]);
    }
    const int wmax = width > n_out ? width : n_out;
    st |= mlp_alloc(h, (void**)&h->G, sizeof(float) * R * wmax);
    st |= mlp_alloc(h, (void**)&h->G2, sizeof(float) * R * wmax);
    st |= mlp_alloc(h, (void**)&h->Gb, sizeof(__nv_bfloat16) * R * wmax);
    st |= mlp_alloc(h, (void**)&h->ws, sizeof(float) * kMaxSplit * (size_t)wmax * (width > n_in ? width : n_in));
    st |= mlp_alloc(h, (void**)&h->x, sizeof(float) * max_batch * n_in);
    st |= mlp_alloc(h, (void**)&h->t, sizeof(float) * max_batch * n_out);
    st |= mlp_alloc(h, (void**)&h->dt, sizeof(float) * max_batch * n_out * n_in);
    st |= mlp_alloc(h, (void**)&h->loss, sizeof(double));
    st |= mlp_alloc(h, (void**)&h->ctr, sizeof(int64_t) * 3);
    st |= mlp_alloc(h, (void**)&h->done, sizeof(unsigned));
    if (st) {
        ad_pic_mlp_destroy(h);
        return AD_PIC_ERR_OOM;
    }
    cudaMemsetAsync(h->p, 0, sizeof(float) * h->n_params, h->stream);
    cudaMemsetAsync(h->m, 0, sizeof(float) * h->n_params, h->stream);
    cudaMemsetAsync(h->v, 0, sizeof(float) * h->n_params, h->stream);
    cudaMemsetAsync(h->pb, 0, sizeof(__nv_bfloat16) * h->n_params, h->stream);
    cudaMemsetAsync(h->ctr, 0, sizeof(int64_t) * 3, h->stream);
    cudaMemsetAsync(h->done, 0, sizeof(unsigned), h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        ad_pic_mlp_destroy(h);
        return AD_PIC_ERR_CUDA;
    }
    *out = h;
    return AD_PIC_OK;
}

int ad_pic_mlp_num_params(const ad_pic_mlp* h, int64_t* n) {
    if (!h || !n) return AD_PIC_ERR_INVALID_ARG;
    *n = h->n_params;
    return AD_PIC_OK;
}

int ad_pic_mlp_set_params(ad_pic_mlp* h, const float* params) {
    if (!h || !params) return AD_PIC_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->p, params, sizeof(float) * h->n_params, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    to_bf16_kernel<<<nb(h->n_params), 256, 0, s>>>(h->p, h->pb, h->n_params);
    cudaMemsetAsync(h->m, 0, sizeof(float) * h->n_params, s);
    cudaMemsetAsync(h->v, 0, sizeof(float) * h->n_params, s);
    cudaMemsetAsync(h->ctr, 0, sizeof(int64_t) * 3, s);
    h->step = 0;
    return cudaStreamSynchronize(s) == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

int ad_pic_mlp_set_dataset(ad_pic_mlp* h, const float* x, const float* t, const float* dt, int n) {
    if (!h || !x || !t || !dt || n < 1) return AD_PIC_ERR_INVALID_ARG;
    if (n > h->data_cap) {
        for (float** q : {&h->dx, &h->dtg, &h->ddt})
            if (*q) {
                cudaFree(*q);
                for (auto& a : h->allocs) if (a == *q) a = nullptr;
                *q = nullptr;
            }
        int st = 0;
        st |= mlp_alloc(h, (void**)&h->dx, sizeof(float) * (size_t)n * h->n_in);
        st |= mlp_alloc(h, (void**)&h->dtg, sizeof(float) * (size_t)n * h->n_out);
        st |= mlp_alloc(h, (void**)&h->ddt, sizeof(float) * (size_t)n * h->n_out * h->n_in);
        if (st) { h->data_cap = 0; return AD_PIC_ERR_OOM; }
        h->data_cap = n;
    }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->dx, x, sizeof(float) * (size_t)n * h->n_in, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->dtg, t, sizeof(float) * (size_t)n * h->n_out, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->ddt, dt, sizeof(float) * (size_t)n * h->n_out * h->n_in, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return AD_PIC_ERR_CUDA;
    h->n_data = n;
    cudaMemsetAsync(h->ctr + 2, 0, sizeof(int64_t), s);
    return cudaStreamSynchronize(s) == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

int ad_pic_mlp_get_params(const ad_pic_mlp* h, float* params) {
    if (!h || !params) return AD_PIC_ERR_INVALID_ARG;
    if (cudaMemcpy(params, h->p, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    return AD_PIC_OK;
}

int ad_pic_mlp_forward(ad_pic_mlp* h, const float* x, int B, float* y, float* dy) {
    if (!h || !x || !y || B < 1 || B > h->max_batch) return AD_PIC_ERR_INVALID_ARG;
    int st = upload(h, x, nullptr, nullptr, B);
    if (st) return st;
    forward_rows(h, B);
    const int S = h->S, n_out = h->n_out;
    std::vector<float> Y((size_t)B * S * n_out);
    if (cudaMemcpyAsync(Y.data(), h->H[h->layers - 1], sizeof(float) * Y.size(), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < n_out; ++o) {
            y[b * n_out + o] = Y[((size_t)b * S) * n_out + o];
            if (dy)
                for (int k = 0; k < h->n_in; ++k)
                    dy[((size_t)b * n_out + o) * h->n_in + k] = Y[((size_t)b * S + 1 + k) * n_out + o];
        }
    return AD_PIC_OK;
}

int ad_pic_mlp_loss_grad(ad_pic_mlp* h, const float* x, const float* t, const float* dt, int B, float lam, double* loss,
                         float* grad) {
    if (!h || !x || !t || !dt || B < 1 || B > h->max_batch || !(lam >= 0.f)) return AD_PIC_ERR_INVALID_ARG;
    int st = upload(h, x, t, dt, B);
    if (st) return st;
    loss_grad(h, B, lam);
    if (loss && cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    if (grad && cudaMemcpyAsync(grad, h->g, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost, h->stream) !=
                    cudaSuccess)
        return AD_PIC_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

int ad_pic_mlp_adam_step(ad_pic_mlp* h, const float* x, const float* t, const float* dt, int B, float lam, float lr,
                         double* loss) {
    if (!h || !x || !t || !dt || B < 1 || B > h->max_batch || !(lam >= 0.f) || !(lr > 0.f)) return AD_PIC_ERR_INVALID_ARG;
    int st = upload(h, x, t, dt, B);
    if (st) return st;
    loss_grad(h, B, lam);
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->step), c2 = 1.f - std::pow(b2, (float)h->step);
    adam_kernel<<<nb(h->n_params), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->pb, h->n_params, lr, b1, b2, 1e-8f,
                                                         c1, c2);
    // Adam's step count on the device follows (ad_pic_mlp_train continues from it)
    const int64_t cnt = h->step;
    cudaMemcpyAsync(h->ctr, &cnt, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
    if (loss && cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

int ad_pic_mlp_train(ad_pic_mlp* h, int steps, int B, float lam, float lr0, float lr1, double* loss, double* ms) {
    if (!h || steps < 1 || B < 1 || B > h->max_batch || !(lam >= 0.f) || !(lr0 > 0.f) || !(lr1 > 0.f))
        return AD_PIC_ERR_INVALID_ARG;
    if (h->n_data < 1) return AD_PIC_ERR_STATE;
    cudaStream_t s = h->stream;
    // one Adam step on the next mini-batch, captured once per (B, lambda, schedule) and replayed
    if (!h->train_graph || h->g_B != B || h->g_lam != lam || h->g_lr0 != lr0 || h->g_lr1 != lr1 ||
        h->g_total != steps) {
        if (h->train_graph) cudaGraphExecDestroy(h->train_graph);
        h->train_graph = nullptr;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AD_PIC_ERR_CUDA;
        const int per = h->n_in + h->n_out + h->n_out * h->n_in;
        gather_batch_kernel<<<nb((int64_t)B * per), 256, 0, s>>>(h->dx, h->dtg, h->ddt, h->n_data, B, h->n_in,
                                                                 h->n_out, h->ctr, h->x, h->t, h->dt);
        loss_grad(h, B, lam);
        adam_dev_kernel<<<nb(h->n_params), 256, 0, s>>>(h->p, h->g, h->m, h->v, h->pb, h->n_params, lr0, lr1, steps,
                                                        0.9f, 0.999f, 1e-8f, h->ctr, h->done);
        if (cudaStreamEndCapture(s, &graph) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_CUDA; }
        const cudaError_t e = cudaGraphInstantiate(&h->train_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { cudaGetLastError(); h->train_graph = nullptr; return AD_PIC_ERR_CUDA; }
        h->g_B = B; h->g_lam = lam; h->g_lr0 = lr0; h->g_lr1 = lr1; h->g_total = steps;
    }
    // the step within this run restarts at 0 (the learning-rate schedule); Adam's count continues
    if (cudaMemsetAsync(h->ctr + 1, 0, sizeof(int64_t), s) != cudaSuccess) return AD_PIC_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int rc = AD_PIC_OK;
    for (int i = 0; i < steps && !rc; ++i)
        if (cudaGraphLaunch(h->train_graph, s) != cudaSuccess) rc = AD_PIC_ERR_CUDA;
    cudaEventRecord(e1, s);
    if (!rc && loss && cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = AD_PIC_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = AD_PIC_ERR_CUDA;
    float t = 0.f;
    if (!rc) cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->step += steps;
    if (rc) cudaGetLastError();
    return rc;
}

void ad_pic_mlp_destroy(ad_pic_mlp* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->train_graph) cudaGraphExecDestroy(h->train_graph);
    for (void* p : h->allocs) cudaFree(p);
    if (h->stream) cudaStreamDestroy(h->stream);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
