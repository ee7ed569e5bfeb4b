// Device code of particles.cu (helpers, kernel bodies taking an explicit block index,
// and their kernel wrappers), shared by particles.cu and the batched persistent kernel.
#pragma once
// Particle kernels: initial distribution, state conversion, the fused
// gather + kick + push (M2 then M1 maps), the period-boundary kernel (dual
// moments in FP64 + half map), and cloud-in-cell deposition of every dual
// channel.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "field_dev.cuh"

namespace adpic {

// ------------------------------------------------------------------ helpers



__device__ __forceinline__ unsigned int ord_enc(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long ord_enc(double f) {
    unsigned long long u = (unsigned long long)__double_as_longlong(f);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

template <typename T>
__device__ __forceinline__ T tmax() { return sizeof(T) == 4 ? (T)FLT_MAX : (T)DBL_MAX; }

// Block-wide min/max of three values, then one atomic per block and quantity.
template <typename T>
__device__ void block_minmax(T (&mn)[3], T (&mx)[3], Ord<T>* mm) {
    __shared__ T smn[32][3], smx[32][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
        for (int d = 0; d < 3; ++d) { smn[w][d] = mn[d]; smx[w][d] = mx[d]; }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T a = l < nw ? smn[l][d] : tmax<T>();
            T b = l < nw ? smx[l][d] : -tmax<T>();
            for (int o = 16; o > 0; o >>= 1) {
                a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
                b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
            }
            if (l == 0 && a <= b) {
                atomicMin(&mm[d], ord_enc(a));
                atomicMax(&mm[3 + d], ord_enc(b));
            }
        }
    }
}

// Cell index and fractional offset of one coordinate; flags and clamps a
// particle outside the stencil range [1, n-3] (the geometry guarantees it).
template <typename T>
__device__ __forceinline__ int cell_of(T x, T o, T ih, int n, T& f, int& bad) {
    T u = (x - o) * ih;
    T fl = floor(u);
    int i = (int)fl;
    if (!(fl >= (T)1 && fl <= (T)(n - 3))) {
        bad |= isfinite(x) ? kErrOutOfGrid : kErrNonfinite;
        i = i < 1 ? 1 : (i > n - 3 ? n - 3 : i);
        if (!isfinite(x)) i = 1;
        fl = (T)i;
        u = fmin(fmax(u, fl), fl + (T)1);
        if (!isfinite(x)) u = fl;
    }
    f = u - fl;
    return i;
}

template <typename T> __device__ __forceinline__ T geom_o(const GeomDev& g, int d) {
    return sizeof(T) == 4 ? (T)g.of[d] : (T)g.o[d];
}
template <typename T> __device__ __forceinline__ T geom_ih(const GeomDev& g, int d) {
    return sizeof(T) == 4 ? (T)g.ihf[d] : (T)g.ihd[d];
}

// ------------------------------------------------------------------ init / convert

// coef [3 planes][3 (a, b, alpha)][CP] duals then 6 means of the normals.
// Per plane: u = a (n1 - mean n1), p = b ((n2 - mean n2) - alpha (n1 - mean n1)).
template <typename T, int C, int CP>
__device__ __forceinline__ void init_kernel_body(const double* __restrict__ nrm, int64_t N, const double* __restrict__ coef,
                            T* __restrict__ state,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    int64_t i = bx_ * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* means = coef + 3 * 3 * CP;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        const double* a = coef + (pl * 3 + 0) * CP;
        const double* b = coef + (pl * 3 + 1) * CP;
        const double* al = coef + (pl * 3 + 2) * CP;
        double n1 = nrm[(2 * pl) * N + i] - means[2 * pl];
        double n2 = nrm[(2 * pl + 1) * N + i] - means[2 * pl + 1];
        double s0 = n2 - al[0] * n1;
        T u[CP], p[CP];
        u[0] = (T)(a[0] * n1);
        p[0] = (T)(b[0] * s0);
#pragma unroll
        for (int k = 1; k < CP; ++k) {
            u[k] = (T)(a[k] * n1);
            p[k] = (T)(b[0] * (-al[k] * n1) + b[k] * s0);
        }
        stg_v<T, CP>(state + ((2 * pl) * N + i) * CP, u);
        stg_v<T, CP>(state + ((2 * pl + 1) * N + i) * CP, p);
    }
}

template <typename T, int C, int CP>
static __global__ void init_kernel(const double* __restrict__ nrm, int64_t N, const double* __restrict__ coef,
                            T* __restrict__ state) {
    init_kernel_body<T, C, CP>(nrm, N, coef, state, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

template <typename T, int CP>
__device__ __forceinline__ void convert_in_kernel_body(const double* __restrict__ src, T* __restrict__ dst, int64_t rows, int C,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    int64_t t = bx_ * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows * CP) return;
    int64_t r = t / CP;
    int k = (int)(t % CP);
    dst[t] = k < C ? (T)src[r * C + k] : (T)0;
}

template <typename T, int CP>
static __global__ void convert_in_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t rows, int C) {
    convert_in_kernel_body<T, CP>(src, dst, rows, C, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

template <typename T, int CP>
__device__ __forceinline__ void convert_out_kernel_body(const T* __restrict__ src, double* __restrict__ dst, int64_t rows, int C,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    int64_t t = bx_ * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows * C) return;
    int64_t r = t / C;
    int k = (int)(t % C);
    dst[t] = (double)src[r * CP + k];
}

template <typename T, int CP>
static __global__ void convert_out_kernel(const T* __restrict__ src, double* __restrict__ dst, int64_t rows, int C) {
    convert_out_kernel_body<T, CP>(src, dst, rows, C, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// ------------------------------------------------------------------ gather + kick + push

// One thread per particle: CIC gather of the dual rest-frame field (the weight
// derivatives carry the particle's derivative channels), the kick M2(tau)
// p += (kappa tau) E (dual product), then the dual map A (one half map, or
// the composition of this kick's and the next kick's half maps), and the
// value-part extrema of the new positions for the next grid geometry.
// The gather runs one field component at a time over the eight nodes, so
// only that component's CP accumulators and its three interpolant gradients
// are live: E_p,k = sum W E_k + sum_d (x_d,k / h_d) sum dW/du_d E_0 (Eq. 2 on
// the weight product), then p_k += a0 E_p,k + a_k E_p,0 in one rounding.

// Where the eight node records of a particle's cell come from: the field
// grid in global memory (read-only path) or a copy of the cell's stencil in
// shared memory (nodes a + 2b + 4c, each 3 x CP values).
template <typename T, int CP>
struct GlobalStencil {
    const T* e0;              // node (0, 0, 0) of the cell
    int64_t sy, sz;           // node strides in y and z (values)
    __device__ __forceinline__ void load(int a, int b, int c, int q, T (&v)[CP]) const {
        ldg_v<T, CP>(e0 + c * sz + b * sy + a * 3 * CP + q * CP, v);
    }
};
template <typename T, int CP>
struct SharedStencil {
    const T* w;               // the cell's stencil copy
    __device__ __forceinline__ void load(int a, int b, int c, int q, T (&v)[CP]) const {
        ldv<T, CP>(w + (a + 2 * b + 4 * c) * 3 * CP + q * CP, v);
    }
};

// cell indices and in-cell offsets of one particle (value part); flags a
// particle outside the stencil range (the index is clamped)
template <typename T>
__device__ __forceinline__ int locate(const T* x, const T* y, const T* z, const GeomDev& g, int nx, int ny, int nz,
                                      int (&idx)[3], T (&f)[3], T (&ih)[3], int& bad) {
    const int n[3] = {nx, ny, nz};
    const T* c[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ih[d] = geom_ih<T>(g, d);
        idx[d] = cell_of<T>(c[d][0], geom_o<T>(g, d), ih[d], n[d], f[d], bad);
    }
    return (idx[2] * ny + idx[1]) * nx + idx[0];
}

// gather of the dual field at the particle and the kick M2(tau)
template <typename T, int C, int CP, typename Src>
__device__ __forceinline__ void kick_core(T (&u)[6][CP], const T (&f)[3], const T (&ih)[3], const Src& src,
                                          const KickCoef<T, CP>& K) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        T Ev[CP];
        T gx = (T)0, gy = (T)0, gz = (T)0;
#pragma unroll
        for (int k = 0; k < CP; ++k) Ev[k] = (T)0;
        // nodes nd = a + 2b + 4c in batches: a batch's loads are all issued before
        // its accumulation, so one round trip serves NB nodes
        constexpr int NB = (CP * sizeof(T) <= 32) ? 4 : 2;
#pragma unroll
        for (int nb0 = 0; nb0 < 8; nb0 += NB) {
            T en[NB][CP];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const int nd = nb0 + j;
                src.load(nd & 1, (nd >> 1) & 1, nd >> 2, q, en[j]);
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const int nd = nb0 + j, a = nd & 1, b = (nd >> 1) & 1, c = nd >> 2;
                const T wz = c ? f[2] : (T)1 - f[2];
                const T sz_ = c ? (T)1 : (T)-1;
                const T wy = b ? f[1] : (T)1 - f[1];
                const T sy_ = b ? (T)1 : (T)-1;
                const T wx = a ? f[0] : (T)1 - f[0];
                const T sx_ = a ? (T)1 : (T)-1;
                const T W = wx * wy * wz;
#pragma unroll
                for (int k = 0; k < CP; ++k) Ev[k] = fma(W, en[j][k], Ev[k]);
                gx = fma(sx_ * wy * wz, en[j][0], gx);
                gy = fma(wx * sy_ * wz, en[j][0], gy);
                gz = fma(wx * wy * sz_, en[j][0], gz);
            }
        }
        gx *= ih[0];
        gy *= ih[1];
        gz *= ih[2];
        T* p = u[2 * q + 1];
        const T a0 = K.a[q][0], E0 = Ev[0];
#pragma unroll
        for (int k = 1; k < CP; ++k) {
            const T Ek = fma(u[0][k], gx, fma(u[2][k], gy, fma(u[4][k], gz, Ev[k])));
            p[k] = fma(a0, Ek, fma(K.a[q][k], E0, p[k]));
        }
        p[0] = fma(a0, E0, p[0]);
    }
}

// the dual map A of every plane
template <typename T, int CP>
__device__ __forceinline__ void map_core(T (&u)[6][CP], const MapCoef<T, CP>& A) {
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        T* x = u[2 * pl];
        T* p = u[2 * pl + 1];
        const T a0 = A.m[pl][0][0], b0 = A.m[pl][1][0], c0 = A.m[pl][2][0], d0 = A.m[pl][3][0];
        const T x0 = x[0], p0 = p[0];
#pragma unroll
        for (int k = 1; k < CP; ++k) {
            const T xk = x[k], pk = p[k];
            x[k] = fma(a0, xk, fma(b0, pk, fma(A.m[pl][0][k], x0, A.m[pl][1][k] * p0)));
            p[k] = fma(c0, xk, fma(d0, pk, fma(A.m[pl][2][k], x0, A.m[pl][3][k] * p0)));
        }
        x[0] = fma(a0, x0, b0 * p0);
        p[0] = fma(c0, x0, d0 * p0);
    }
}

// Gather + kick + dual map of one particle held in registers (u[6][CP]), field
// records read from global memory.
template <typename T, int C, int CP>
__device__ __forceinline__ void push_core(T (&u)[6][CP], const T* __restrict__ E, const GeomDev* __restrict__ geom,
                                          int nx, int ny, int nz, const MapCoef<T, CP>& A, const KickCoef<T, CP>& K,
                                          int* __restrict__ err) {
    if (E != nullptr) {
        int idx[3];
        T f[3], ih[3];
        int bad = 0;
        locate<T>(u[0], u[2], u[4], *geom, nx, ny, nz, idx, f, ih, bad);
        if (bad) atomicOr(err, bad);
        GlobalStencil<T, CP> src;
        src.e0 = E + (((int64_t)idx[2] * ny + idx[1]) * nx + idx[0]) * (3 * CP);
        src.sy = (int64_t)nx * 3 * CP;
        src.sz = (int64_t)nx * ny * 3 * CP;
        kick_core<T, C, CP>(u, f, ih, src, K);
    }
    map_core<T, CP>(u, A);
}

template <typename T, int C, int CP, bool TRACK>
__device__ __forceinline__ void push_kernel_body(const T* __restrict__ state, T* __restrict__ out, int64_t N, const T* __restrict__ E,
                const GeomDev* __restrict__ geom, int nx, int ny, int nz, const MapCoef<T, CP>& A,
                const KickCoef<T, CP>& K, Ord<T>* __restrict__ mm, int* __restrict__ err, const SortBuf sb,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int64_t t = bx_ * (int64_t)blockDim.x + threadIdx.x;
    T mn[3] = {tmax<T>(), tmax<T>(), tmax<T>()};
    T mx[3] = {-tmax<T>(), -tmax<T>(), -tmax<T>()};
    if (t < N) {
        // particle i to slot dst (see SortBuf)
        const int64_t i = t;
        const int64_t dst = sb.offs ? (int64_t)sb.offs[sb.key[i]] + sb.rank[i] : i;
        T u[6][CP];
#pragma unroll
        for (int c = 0; c < 6; ++c) ldg_v<T, CP>(state + (c * N + i) * CP, u[c]);
        push_core<T, C, CP>(u, E, geom, nx, ny, nz, A, K, err);
        if (sb.ids_out) sb.ids_out[dst] = sb.ids_in[i];
#pragma unroll
        for (int c = 0; c < 6; ++c) stg_v<T, CP>(out + (c * N + dst) * CP, u[c]);
        if (TRACK) {
#pragma unroll
            for (int d = 0; d < 3; ++d) { mn[d] = u[2 * d][0]; mx[d] = u[2 * d][0]; }
        }
    }
    if (TRACK) block_minmax<T>(mn, mx, mm);
}


// ------------------------------------------------------------------ push over bulk-copied tiles

// Shared-memory barrier and bulk-copy primitives (PTX). A tile copy is six
// contiguous runs (one per coordinate) of TP particles' dual records.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: gives up after `polls` failed polls (0: at once, without polling).
// Each failed try_wait suspends the thread for a system-dependent time, about
// 1.9 us measured on GB300 (ad_pic_wait_probe), so the default limit of 2^18
// polls gives up after about half a second; a tile copy lands within microseconds
constexpr int kWaitPolls = 1 << 18;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int polls = kWaitPolls) {
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// particles per tile (one thread each) and resident CTAs per SM the register
// budget is sized for: 2 KB coordinate runs and six 64-thread CTAs for the
// 32-byte records (168 registers, no spills; two warps per tile barrier); 4 KB
// runs and four 64-thread CTAs for the FP32 64-byte records (255 registers:
// the 8 warps per SM of two 128-thread CTAs, with two warps per tile barrier);
// 8 KB runs and two CTAs otherwise
template <typename T, int CP>
__host__ __device__ constexpr int push_tile() {
    return (CP * sizeof(T) == 32 || (sizeof(T) == 4 && CP == 16)) ? 64 : (int)(8192 / (CP * sizeof(T)));
}
template <typename T, int CP>
__host__ __device__ constexpr int push_min_blocks() {
    return CP * sizeof(T) == 32 ? 6 : ((sizeof(T) == 4 && CP == 16) ? 4 : 2);
}
// Field stencils staged in shared memory per warp and tile (FP32, P = 7): the
// distinct cells of a warp's particles, up to this many, each as its eight
// node records (3 x CP values each) plus 16 bytes of padding, so stencils of
// different cells start in different banks
template <typename T, int CP>
__host__ __device__ constexpr int push_window_slots() {
    return (sizeof(T) == 4 && CP == 8) ? 6 : 0;
}
template <typename T, int CP>
__host__ __device__ constexpr int push_window_stride() {
    return 8 * 3 * CP + (int)(16 / sizeof(T));
}
// dynamic shared memory of the persistent push: the two-stage state ring and
// the warps' stencil windows
template <typename T, int CP>
__host__ __device__ constexpr size_t push_smem() {
    return sizeof(T) * ((size_t)2 * 6 * push_tile<T, CP>() * CP +
                        (size_t)(push_tile<T, CP>() / 32) * push_window_slots<T, CP>() * push_window_stride<T, CP>()) +
           sizeof(int) * (size_t)2 * 2 * push_tile<T, CP>();     // each stage's slots and ids
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Persistent push: each CTA walks tiles blockIdx.x, +gridDim.x, ... and keeps
// two tiles of the dual state in flight in a two-stage shared-memory ring
// (one mbarrier per stage), so the DRAM reads run ahead of the gather and
// the map without holding registers. One thread per particle of a tile; the
// results go to their cell-sorted slots as in push_kernel. Every wait is
// bounded; the CTA agrees on the outcome with a barrier vote, and on a timeout
// it records kErrTimeout, lets its copies land (bounded) and stops.
// With stencil windows (push_window_slots > 0) each warp finds the distinct
// cells of its particles (the particles are sorted by cell, so a warp holds
// few), copies each cell's eight node records once into shared memory with
// asynchronous copies, all in flight together, and gathers from there: one
// round trip to L2 per warp and tile instead of several per particle. A
// particle whose cell got no slot gathers from global memory.
template <typename T, int C, int CP, bool TRACK>
__device__ __forceinline__ void push_tma_body(const T* __restrict__ state, T* __restrict__ out, int64_t N,
                                              const T* __restrict__ E, const GeomDev* __restrict__ geom, int nx,
                                              int ny, int nz, const MapCoef<T, CP>& A, const KickCoef<T, CP>& K,
                                              Ord<T>* __restrict__ mm, int* __restrict__ err, const SortBuf sb,
                                              int polls = kWaitPolls) {
    constexpr int TP = push_tile<T, CP>();
    constexpr int KW = push_window_slots<T, CP>();
    constexpr int WS = push_window_stride<T, CP>();
    constexpr int PPN = 3 * CP * (int)sizeof(T) / 16;       // 16-byte pieces per node record
    extern __shared__ __align__(128) unsigned char smraw[];
    T* ring = reinterpret_cast<T*>(smraw);      // [2][6][TP][CP]
    int* aux = reinterpret_cast<int*>(ring + (size_t)2 * 6 * TP * CP);   // [2][2][TP]: slots, ids
    T* win = reinterpret_cast<T*>(aux + 2 * 2 * TP);                      // [TP / 32][KW][WS]
    __shared__ int s_cell[TP / 32][KW > 0 ? KW : 1];
    __shared__ int s_slot[TP], s_id[TP];        // this tile's slots and ids, kept past the ring's reuse
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int64_t ntiles = (N + TP - 1) / TP;
    const int64_t step = gridDim.x;
    // the slots (sb.dst, required) and ids travel with the state
    auto issue = [&](int64_t tl, int s) {
        const int64_t p0 = tl * TP;
        const int n = (int)min((int64_t)TP, N - p0);
        const unsigned bytes = (unsigned)n * CP * (unsigned)sizeof(T);
        // slot and id runs rounded up to 16 bytes (the arrays are padded by 4 entries)
        const unsigned ib = ((unsigned)n * 4u + 15u) & ~15u;
        mbar_expect_tx(&bar[s], 6u * bytes + 2u * ib);
#pragma unroll
        for (int c = 0; c < 6; ++c)
            bulk_g2s(ring + ((size_t)(s * 6 + c) * TP) * CP, state + ((size_t)c * N + p0) * CP, bytes, &bar[s]);
        bulk_g2s(aux + (s * 2 + 0) * TP, sb.dst + p0, ib, &bar[s]);
        bulk_g2s(aux + (s * 2 + 1) * TP, sb.ids_in + p0, ib, &bar[s]);
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int64_t tile = blockIdx.x;
    if (tid == 0) {
        if (tile < ntiles) issue(tile, 0);
        if (tile + step < ntiles) issue(tile + step, 1);
    }
    T mn[3] = {tmax<T>(), tmax<T>(), tmax<T>()};
    T mx[3] = {-tmax<T>(), -tmax<T>(), -tmax<T>()};
    int it = 0;
    bool ok = true;
    for (; tile < ntiles; tile += step, ++it) {
        const int s = it & 1;
        const bool got = mbar_wait(&bar[s], (unsigned)((it >> 1) & 1), polls);
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        const int64_t i = tile * TP + tid;
        const bool valid = i < N;
        const T* row = ring + ((size_t)s * 6 * TP + tid) * CP;     // coordinate c at row + c * TP * CP
        // stencil windows: the cells from the value parts alone, and the copies of
        // the distinct cells' stencils issued before the state goes to registers
        int L = -1, slot = 0, bad = 0;
        T f[3], ih[3];
        const bool win_on = KW > 0 && E != nullptr;
        if constexpr (KW > 0) {
            if (win_on) {
                const int lane = tid & 31, warp = tid >> 5;
                int idx[3];
                if (valid) L = locate<T>(row, row + 2 * TP * CP, row + 4 * TP * CP, *geom, nx, ny, nz, idx, f, ih, bad);
                // the warp's distinct cells: the lowest lane of each cell owns a slot
                const unsigned match = __match_any_sync(0xffffffffu, L);
                const int lead = __ffs(match) - 1;
                const unsigned heads = __ballot_sync(0xffffffffu, valid && lead == lane);
                slot = __popc(heads & ((1u << lead) - 1u));
                const int k = min(__popc(heads), KW);
                __syncwarp();                    // the warp's gathers from its window are done
                if (valid && lead == lane && slot < KW) s_cell[warp][slot] = L;
                __syncwarp();
                const int64_t sy = (int64_t)nx * 3 * CP, sz = (int64_t)nx * ny * 3 * CP;
                T* wwin = win + (size_t)warp * KW * WS;
                // one (stencil, node) pair per lane and trip: the node record's 16-byte pieces
                for (int pr = lane; pr < k * 8; pr += 32) {
                    const int sl = pr >> 3, nd = pr & 7;
                    const T* src = E + (int64_t)s_cell[warp][sl] * (3 * CP) + (nd >> 2) * sz + ((nd >> 1) & 1) * sy +
                                   (nd & 1) * (3 * CP);
                    T* dstw = wwin + sl * WS + nd * 3 * CP;
#pragma unroll
                    for (int pc = 0; pc < PPN; ++pc)
                        cp_async16(dstw + pc * (16 / (int)sizeof(T)), src + pc * (16 / (int)sizeof(T)));
                }
            }
        }
        T u[6][CP];
        if (valid) {
#pragma unroll
            for (int c = 0; c < 6; ++c) ldv<T, CP>(row + (size_t)c * TP * CP, u[c]);
            s_slot[tid] = aux[(s * 2 + 0) * TP + tid];      // slots and ids are 32-bit: N < 2^31
            s_id[tid] = aux[(s * 2 + 1) * TP + tid];
        }
        __syncthreads();                         // stage s is free again
        if (tid == 0 && tile + 2 * step < ntiles) {
            fence_proxy_async_smem();
            issue(tile + 2 * step, s);
        }
        if constexpr (KW > 0) {
            if (win_on) {
                if (bad) atomicOr(err, bad);
                cp_async_wait_all();
                __syncwarp();
                if (valid) {
                    if (slot < KW) {
                        SharedStencil<T, CP> st_;
                        st_.w = win + ((size_t)(tid >> 5) * KW + slot) * WS;
                        kick_core<T, C, CP>(u, f, ih, st_, K);
                    } else {
                        GlobalStencil<T, CP> st_;
                        st_.e0 = E + (int64_t)L * (3 * CP);
                        st_.sy = (int64_t)nx * 3 * CP;
                        st_.sz = (int64_t)nx * ny * 3 * CP;
                        kick_core<T, C, CP>(u, f, ih, st_, K);
                    }
                    map_core<T, CP>(u, A);
                }
            } else if (valid) {
                map_core<T, CP>(u, A);
            }
        } else if (valid) {
            push_core<T, C, CP>(u, E, geom, nx, ny, nz, A, K, err);
        }
        if (valid) {
            const int dst = s_slot[tid];
            sb.ids_out[dst] = s_id[tid];
#pragma unroll
            for (int c = 0; c < 6; ++c) stg_v<T, CP>(out + (c * N + (int64_t)dst) * CP, u[c]);
            if (TRACK) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    mn[d] = fmin(mn[d], u[2 * d][0]);
                    mx[d] = fmax(mx[d], u[2 * d][0]);
                }
            }
        }
    }
    if (!ok && tid == 0) {
        // the copies still in flight land before the CTA exits (default, long limit)
        atomicOr(err, kErrTimeout);
        const int s = it & 1;
        mbar_wait(&bar[s], (unsigned)((it >> 1) & 1));
        if (tile + step < ntiles) mbar_wait(&bar[1 - s], (unsigned)(((it + 1) >> 1) & 1));
    }
    if (TRACK) block_minmax<T>(mn, mx, mm);
}

template <typename T, int C, int CP, bool TRACK>
static __global__ void __launch_bounds__(push_tile<T, CP>(), push_min_blocks<T, CP>())
    push_tma_kernel(const T* __restrict__ state, T* __restrict__ out, int64_t N, const T* __restrict__ E,
                    const GeomDev* __restrict__ geom, int nx, int ny, int nz, const MapCoef<T, CP> A,
                    const KickCoef<T, CP> K, Ord<T>* __restrict__ mm, int* __restrict__ err, const SortBuf sb,
                    const GeomFuse gf, int polls) {
    push_tma_body<T, C, CP, TRACK>(state, out, N, E, geom, nx, ny, nz, A, K, mm, err, sb, polls);
    // every block has finished its gathers before it counts itself done, so the
    // last block may overwrite the geometry they read
    if (TRACK && gf.count) geom_last_block<T>(gf, mm);
}

// ------------------------------------------------------------------ cell sort: scan, ids

constexpr int kScanChunk = 2048;

__device__ __forceinline__ int block_excl_scan(int v, int* sm, int& total) {
    // 256-thread exclusive scan of one int per thread
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sm[lane] = t;
    }
    __syncthreads();
    total = sm[(blockDim.x >> 5) - 1];
    const int before = w > 0 ? sm[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// per-chunk totals of hist
__device__ __forceinline__ void scan_sum_kernel_body(const int* __restrict__ hist, int ncells, int* __restrict__ bsum,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    __shared__ int sm[32];
    const int base = bx_ * kScanChunk;
    int v = 0;
    for (int j = threadIdx.x; j < kScanChunk; j += blockDim.x)
        if (base + j < ncells) v += hist[base + j];
    int total;
    block_excl_scan(v, sm, total);
    if (threadIdx.x == 0) bsum[bx_] = total;
}

static __global__ void scan_sum_kernel(const int* __restrict__ hist, int ncells, int* __restrict__ bsum) {
    scan_sum_kernel_body(hist, ncells, bsum, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// exclusive scan of the chunk totals (one block; at most 256 x 8 chunks)
__device__ __forceinline__ void scan_top_kernel_body(int* __restrict__ bsum, int nb,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    __shared__ int sm[32];
    constexpr int PER = 8;
    int v[PER], s = 0;
    for (int q = 0; q < PER; ++q) {
        const int j = threadIdx.x * PER + q;
        v[q] = j < nb ? bsum[j] : 0;
        s += v[q];
    }
    int total;
    int run = block_excl_scan(s, sm, total);
    for (int q = 0; q < PER; ++q) {
        const int j = threadIdx.x * PER + q;
        if (j < nb) bsum[j] = run;
        run += v[q];
    }
}


// exclusive offsets of every cell; clears hist for the next kick. With
// `prefixed` bsum holds the exclusive prefixes of the chunk totals (scan_top
// ran); otherwise it holds the totals and each block sums those before it.
__device__ __forceinline__ void scan_apply_kernel_body(int* __restrict__ hist, int ncells, const int* __restrict__ bsum,
                                  int* __restrict__ offs,
    const int bx_, const int by_, const int bz_, const int nbx_, bool prefixed = true) {
    __shared__ int sm[32];
    constexpr int PER = kScanChunk / 256;
    const int base = bx_ * kScanChunk + threadIdx.x * PER;
    int before;
    if (prefixed) {
        before = bsum[bx_];
    } else {
        int t = 0;
        for (int b = threadIdx.x; b < bx_; b += blockDim.x) t += bsum[b];
        int tot;
        block_excl_scan(t, sm, tot);
        before = tot;
    }
    int v[PER], s = 0;
    for (int q = 0; q < PER; ++q) {
        v[q] = base + q < ncells ? hist[base + q] : 0;
        s += v[q];
    }
    int total;
    int run = block_excl_scan(s, sm, total) + before;
    for (int q = 0; q < PER; ++q) {
        if (base + q < ncells) {
            offs[base + q] = run;
            hist[base + q] = 0;
        }
        run += v[q];
    }
}

static __global__ void scan_apply_kernel(int* __restrict__ hist, int ncells, const int* __restrict__ bsum,
                                  int* __restrict__ offs) {
    scan_apply_kernel_body(hist, ncells, bsum, offs, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x,
                           false);
}

static __global__ void slots_kernel(const int* __restrict__ key, const int* __restrict__ rank,
                                    const int* __restrict__ offs, int* __restrict__ dst, int64_t N) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) dst[i] = offs[key[i]] + rank[i];
}

__device__ __forceinline__ void iota_kernel_body(int* ids, int64_t N,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int64_t i = bx_ * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) ids[i] = (int)i;
}

static __global__ void iota_kernel(int* ids, int64_t N) {
    iota_kernel_body(ids, N, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// device state [6][N][CP] in sorted order -> host layout [6][N][C] in the caller's order
template <typename T, int CP>
__device__ __forceinline__ void convert_out_perm_kernel_body(const T* __restrict__ src, const int* __restrict__ ids, double* __restrict__ dst,
                                        int64_t N, int C,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int64_t t = bx_ * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 6 * N * C) return;
    const int k = (int)(t % C);
    const int64_t i = (t / C) % N, c = t / ((int64_t)N * C);
    dst[(c * N + ids[i]) * C + k] = (double)src[(c * N + i) * CP + k];
}

template <typename T, int CP>
static __global__ void convert_out_perm_kernel(const T* __restrict__ src, const int* __restrict__ ids, double* __restrict__ dst,
                                        int64_t N, int C) {
    convert_out_perm_kernel_body<T, CP>(src, ids, dst, N, C, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// ------------------------------------------------------------------ half map alone

// The dual half map A applied in place to every particle (one thread per
// particle, 32-byte loads and stores), with the value-part extrema of the new
// positions for the next grid geometry: the opening pass of a run.
template <typename T, int C, int CP>
static __global__ void __launch_bounds__(256) halfmap_kernel(T* __restrict__ state, int64_t N, const MapCoef<T, CP> A,
                                                             Ord<T>* __restrict__ mm, const GeomFuse gf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    T mn[3] = {tmax<T>(), tmax<T>(), tmax<T>()};
    T mx[3] = {-tmax<T>(), -tmax<T>(), -tmax<T>()};
    if (i < N) {
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            T x[CP], p[CP];
            ldr_v<T, CP>(state + ((2 * pl) * N + i) * CP, x);
            ldr_v<T, CP>(state + ((2 * pl + 1) * N + i) * CP, p);
            const T a0 = A.m[pl][0][0], b0 = A.m[pl][1][0], c0 = A.m[pl][2][0], d0 = A.m[pl][3][0];
            const T x0 = x[0], p0 = p[0];
#pragma unroll
            for (int k = 1; k < CP; ++k) {
                const T xk = x[k], pk = p[k];
                x[k] = fma(a0, xk, fma(b0, pk, fma(A.m[pl][0][k], x0, A.m[pl][1][k] * p0)));
                p[k] = fma(c0, xk, fma(d0, pk, fma(A.m[pl][2][k], x0, A.m[pl][3][k] * p0)));
            }
            x[0] = fma(a0, x0, b0 * p0);
            p[0] = fma(c0, x0, d0 * p0);
            stg_v<T, CP>(state + ((2 * pl) * N + i) * CP, x);
            stg_v<T, CP>(state + ((2 * pl + 1) * N + i) * CP, p);
            mn[pl] = x[0];
            mx[pl] = x[0];
        }
    }
    block_minmax<T>(mn, mx, mm);
    if (gf.count) geom_last_block<T>(gf, mm);
}

// ------------------------------------------------------------------ period boundary: moments + half map

// CP lanes per particle, lane k holds channel k of every coordinate. Each lane
// accumulates, in FP64, channel k of the dual sums of u, p, u^2, u p, p^2
// per plane (Eq. 2 for the products: d(u^2) = 2 u u_k, d(u p) = u p_k + p u_k),
// and optionally applies the dual half map A to the state and tracks extrema.
// Error-free transformations (Knuth's TwoSum, the FMA-based TwoProduct) on an
// unevaluated-pair accumulator (hi, lo) of the state's type: the running sum
// is hi + lo and its rounding does not depend on the order of the terms.
template <typename T>
__device__ __forceinline__ void ef_add(T& hi, T& lo, T a) {
    const T s = hi + a;
    const T bb = s - hi;
    const T e = (hi - (s - bb)) + (a - bb);
    hi = s;
    lo += e;
}
// a product the compiler may not contract into a following addition
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ __forceinline__ void ef_add_prod(T& hi, T& lo, T a, T b) {
    const T ph = mul_rn(a, b);
    const T pl = fma(a, b, -ph);
    ef_add(hi, lo, ph);
    lo += pl;
}

constexpr int kBoundaryBlocks = 152 * 8;

template <typename T, int C, int CP, bool MOM, bool APPLY>
__device__ __forceinline__ void boundary_kernel_body(T* __restrict__ state, int64_t N, const MapCoef<T, CP>& A,
                                                       double* __restrict__ partial, Ord<T>* __restrict__ mm,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    constexpr int PPW = 32 / CP;
    const int lane = threadIdx.x & 31;
    const int k = lane & (CP - 1);
    const int src = lane & ~(CP - 1);
    const int64_t warp = (bx_ * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)nbx_ * blockDim.x) >> 5;
    T ah[3][5], al[3][5];       // compensated per-lane sums (hi, lo)
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
#pragma unroll
        for (int q = 0; q < 5; ++q) { ah[pl][q] = (T)0; al[pl][q] = (T)0; }
    T mn[3] = {tmax<T>(), tmax<T>(), tmax<T>()};
    T mx[3] = {-tmax<T>(), -tmax<T>(), -tmax<T>()};
    // four particle groups per trip: their 24 loads are issued before any use
    constexpr int U = 4;
    const int64_t stride = nwarps * PPW;
    for (int64_t base = warp * PPW; base < N; base += U * stride) {
        T uu[U][3], pv[U][3];
        bool vd[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t i = base + j * stride + lane / CP;
            vd[j] = i < N;
#pragma unroll
            for (int pl = 0; pl < 3; ++pl) {
                uu[j][pl] = vd[j] ? state[((2 * pl) * N + i) * CP + k] : (T)0;
                pv[j][pl] = vd[j] ? state[((2 * pl + 1) * N + i) * CP + k] : (T)0;
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
        const int64_t i = base + j * stride + lane / CP;
        const bool valid = vd[j];
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            T* pu = state + ((2 * pl) * N + i) * CP + k;
            T* pp = state + ((2 * pl + 1) * N + i) * CP + k;
            T u = uu[j][pl];
            T p = pv[j][pl];
            T u0 = __shfl_sync(0xffffffffu, u, src);
            T p0 = __shfl_sync(0xffffffffu, p, src);
            if (MOM && valid) {
                // every product is formed exactly as a pair (hi, lo) and added with
                // error-free sums, so a lane's partials carry about twice the
                // state's precision (about 48 bits in FP32, 106 in FP64)
                const T a = (T)2 * u0;
                ef_add(ah[pl][0], al[pl][0], u);
                ef_add(ah[pl][1], al[pl][1], p);
                if (k == 0) {
                    ef_add_prod(ah[pl][2], al[pl][2], u, u);
                    ef_add_prod(ah[pl][3], al[pl][3], u, p);
                    ef_add_prod(ah[pl][4], al[pl][4], p, p);
                } else {
                    ef_add_prod(ah[pl][2], al[pl][2], a, u);
                    ef_add_prod(ah[pl][3], al[pl][3], u0, p);
                    ef_add_prod(ah[pl][3], al[pl][3], p0, u);
                    ef_add_prod(ah[pl][4], al[pl][4], (T)2 * p0, p);
                }
            }
            if (APPLY && valid) {
                const T a0 = A.m[pl][0][0], b0 = A.m[pl][1][0], c0 = A.m[pl][2][0], d0 = A.m[pl][3][0];
                T un, pn;
                if (k == 0) {
                    un = fma(a0, u, b0 * p);
                    pn = fma(c0, u, d0 * p);
                    mn[pl] = fmin(mn[pl], un);
                    mx[pl] = fmax(mx[pl], un);
                } else {
                    un = fma(a0, u, fma(b0, p, fma(A.m[pl][0][k], u0, A.m[pl][1][k] * p0)));
                    pn = fma(c0, u, fma(d0, p, fma(A.m[pl][2][k], u0, A.m[pl][3][k] * p0)));
                }
                *pu = un;
                *pp = pn;
            }
        }
        }
    }
    if (APPLY) block_minmax<T>(mn, mx, mm);
    if (MOM) {
        // compensated sums over the PPW particle groups of the warp (lanes with the
        // same k), then the pairs in FP64 (a float pair converts exactly)
        // (in the state's type: FP64 work is slow on this part, and the float pairs
        // keep their ~48 bits through these few additions)
        double hh[3][5], ll[3][5];
#pragma unroll
        for (int pl = 0; pl < 3; ++pl)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                T h_ = ah[pl][q], l_ = al[pl][q];
                for (int o = CP; o < 32; o <<= 1) {
                    const T oh = __shfl_xor_sync(0xffffffffu, h_, o);
                    const T ol = __shfl_xor_sync(0xffffffffu, l_, o);
                    ef_add(h_, l_, oh);
                    l_ += ol;
                }
                hh[pl][q] = (double)h_;
                ll[pl][q] = (double)l_;
            }
        // a warp's pair is rounded once to FP64 (one rounding of a partial sum, which
        // does not grow with the number of terms); the warps' partials are summed
        // with compensation
        __shared__ double sm[8][15][CP];
        const int w = threadIdx.x >> 5;
        if (lane < CP)
            for (int pl = 0; pl < 3; ++pl)
                for (int q = 0; q < 5; ++q) sm[w][pl * 5 + q][lane] = hh[pl][q] + ll[pl][q];
        __syncthreads();
        for (int t = threadIdx.x; t < 15 * CP; t += blockDim.x) {
            double sh = 0.0, sl = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) ef_add(sh, sl, sm[ww][t / CP][t % CP]);
            partial[(int64_t)bx_ * 15 * CP + t] = sh + sl;
        }
    }
}

template <typename T, int C, int CP, bool MOM, bool APPLY>
static __global__ void __launch_bounds__(256) boundary_kernel(T* __restrict__ state, int64_t N, const MapCoef<T, CP> A,
                                                       double* __restrict__ partial, Ord<T>* __restrict__ mm,
                                                       const GeomFuse gf) {
    boundary_kernel_body<T, C, CP, MOM, APPLY>(state, N, A, partial, mm, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
    if (APPLY && gf.count) geom_last_block<T>(gf, mm);
}

// partial [nblocks][15][CP] -> out [15][CP] / N: one block per output value,
// a fixed strided split (compensated sums) and a fixed shared-memory tree
// (reproducible; eight levels of 256 partials)
__device__ __forceinline__ void moments_reduce_kernel_body(const double* __restrict__ partial, int nblocks, int CP, int64_t N,
                                      double* __restrict__ out,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    __shared__ double sm[256];
    const int t = bx_;            // output index in [0, 15 CP)
    double sh = 0.0, sl = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) ef_add(sh, sl, partial[(int64_t)b * 15 * CP + t]);
    sm[threadIdx.x] = sh + sl;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = N > 0 ? sm[0] / (double)N : 0.0;
}

static __global__ void moments_reduce_kernel(const double* __restrict__ partial, int nblocks, int CP, int64_t N,
                                      double* __restrict__ out) {
    moments_reduce_kernel_body(partial, nblocks, CP, N, out, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}


// ------------------------------------------------------------------ warp-sorted deposition

// row stride of a lane's node records (4 nodes) in the deposit tile (16-byte
// aligned; 4 mod 32 words apart so the vector stores of 8 lanes hit distinct banks)
template <int CP>
__host__ __device__ constexpr int dep_tile_stride() { return 4 * CP + 4; }
template <int CP, typename T>
__host__ __device__ constexpr size_t dep_tile_bytes_per_warp() { return sizeof(T) * 32 * dep_tile_stride<CP>(); }
// resident blocks per SM the deposit's registers are budgeted for
template <typename T, int CP>
__host__ __device__ constexpr int dep_min_blocks() {
    return sizeof(T) == 4 ? (CP == 8 ? 4 : 3) : 2;
}
template <int CP, typename T>
__host__ __device__ constexpr int dep_tile_warps() {
    return (dep_tile_bytes_per_warp<CP, T>() * 8 <= 72 * 1024) ? 8 : ((dep_tile_bytes_per_warp<CP, T>() * 4 <= 72 * 1024) ? 4 : 2);
}

// Deposition with the summation over particles done on chip before the atomics.
// Each warp takes 32 consecutive particles and sorts them by cell with a
// bitonic network on the keys (cell << 5 | lane), so the particles of one cell
// occupy consecutive sorted positions. Every lane keeps its own particle in
// registers. For each z plane of the stencil in turn, it writes its 4 node
// records (4 x CP values) as row (its sorted position) of a per-warp shared
// tile [32][4 CP + 4] with vector stores; then lane j owns tile columns j,
// j + 32, ... (node = column / CP, channel column % CP) and, for each run of
// lanes sharing a cell, sums its columns over the run and issues one scalar
// atomic per (run, node, channel). Consecutive lanes then address consecutive
// channels of neighbouring nodes, so one warp atomic touches a few contiguous
// sectors. The cell sort's rank is the lane's offset in its run plus one
// counting atomic per run.

// QS: the bunch charge Q is the AD variable of slot qslot; channel qslot + 1
// then also gets dq_m/dQ W = W / N (qmd = 1 / N) per node (Eq. 2 on q_m W).
template <typename T, int C, int CP, int WARPS, bool QS = false>
__device__ __forceinline__ void deposit_tile_body(const T* __restrict__ state, int64_t N,
                                                    const GeomDev* __restrict__ geom, int nx, int ny, int nz, T qm,
                                                    T* __restrict__ rho, int* __restrict__ err, const SortBuf sb,
                                                    const int bx_, int qslot = -1, T qmd = (T)0) {
    constexpr int ROWS = 4 * CP;                            // tile columns: 4 nodes x CP
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int RS = dep_tile_stride<CP>();
    T* tile = reinterpret_cast<T*>(smraw) + (size_t)warp * 32 * RS;    // [sorted lane][8 CP (+4)]
    const int64_t i0 = ((int64_t)bx_ * WARPS + warp) * 32;
    if (i0 >= N) return;                                  // whole warp
    const int64_t i = i0 + lane;
    const bool valid = i < N;
    const GeomDev& g = *geom;
    const int n[3] = {nx, ny, nz};
    T ih[3], o[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ih[d] = geom_ih<T>(g, d);
        o[d] = geom_o<T>(g, d);
    }
    int bad = 0;
    // this lane's particle: its x, y, z records stay in registers through the sort
    int key = (0x3ffffff << 5) | lane;                    // invalid lanes sort last
    T f[3] = {(T)0, (T)0, (T)0};
    T x[3][CP];
    if (valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) ldg_v_stream<T, CP>(state + ((2 * d) * N + i) * CP, x[d], l2_evict_first());
        int idx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) idx[d] = cell_of<T>(x[d][0], o[d], ih[d], n[d], f[d], bad);
        key = (((idx[2] * ny + idx[1]) * nx + idx[0]) << 5) | lane;
    }
    // bitonic sort of the 32 (distinct) keys, ascending in lane order; skipped
    // when they already are (slots follow the previous kick's cell order)
    const int next_key = __shfl_down_sync(FULL, key, 1);
    if (!__all_sync(FULL, lane == 31 || key < next_key)) {
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int other = __shfl_xor_sync(FULL, key, j);
                const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                key = (lower == up) ? min(key, other) : max(key, other);
            }
        }
    }
    const int nv = __popc(__ballot_sync(FULL, valid));    // sorted lanes [0, nv) hold particles
    const bool sv = lane < nv;
    const int cell = key >> 5;
    const int src = key & 31;
    const int64_t ps = i0 + src;
    // sorted position of this lane's own particle (sorted lane j holds lane src_j's)
    __shared__ int spos[WARPS][32];
    spos[warp][src] = lane;
    __syncwarp();
    const int mypos = spos[warp][lane];
    // runs of equal cells
    const int prev = __shfl_up_sync(FULL, cell, 1);
    const bool head = sv && (lane == 0 || prev != cell);
    const unsigned heads = __ballot_sync(FULL, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    // the run's counting atomic is issued here and its result consumed after
    // the sums below, so its round trip to L2 overlaps them
    int base = 0;
    if (sb.key) {
        const unsigned after = heads & ~(0xffffffffu >> (31 - lane));
        const int end = after ? __ffs(after) - 2 : nv - 1;
        if (head) base = atomicAdd(&sb.hist[cell], end - lane + 1);
        if (sv) sb.key[ps] = cell;
    }
    // Two halves of the stencil, the nodes of the lower (c = 0) then the upper
    // (c = 1) z plane: the tile holds one half (4 node records per row), so it
    // takes half the shared memory and twice the warps fit on an SM.
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (c) __syncwarp();                              // the lower half's sums are read
        // node records of this lane's particle into tile row `mypos` (sorted order)
        if (valid) {
#pragma unroll
            for (int nb = 0; nb < 4; ++nb) {
                const int a = nb & 1, b = nb >> 1;
                const T wx = a ? f[0] : (T)1 - f[0], sx = a ? (T)1 : (T)-1;
                const T wy = b ? f[1] : (T)1 - f[1], sy = b ? (T)1 : (T)-1;
                const T wz = c ? f[2] : (T)1 - f[2], sz = c ? (T)1 : (T)-1;
                const T gx = qm * ih[0] * sx * wy * wz, gy = qm * ih[1] * wx * sy * wz, gz = qm * ih[2] * wx * wy * sz;
                // rec[k] = x_k gx + y_k gy + z_k gz (k >= 1), lane pairs at once; rec[0] = q W
                T rec[CP];
                const V2<T> gx2 = {gx, gx}, gy2 = {gy, gy}, gz2 = {gz, gz};
#pragma unroll
                for (int k = 0; k < CP; k += 2) {
                    const V2<T> r = v2_fma(V2<T>{x[0][k], x[0][k + 1]}, gx2,
                                           v2_fma(V2<T>{x[1][k], x[1][k + 1]}, gy2,
                                                  v2_mul(V2<T>{x[2][k], x[2][k + 1]}, gz2)));
                    rec[k] = r.x;
                    rec[k + 1] = r.y;
                }
                rec[0] = qm * (wx * wy * wz);
                if constexpr (QS) {
#pragma unroll
                    for (int k = 1; k < CP; ++k)
                        if (k == qslot + 1) rec[k] = fma(qmd, wx * wy * wz, rec[k]);
                }
                stv<T, CP>(tile + mypos * RS + nb * CP, rec);
            }
        }
        __syncwarp();
        // columns of this lane: node nb = r / CP of the half (node index = cell index +
        // offset, as cells and nodes share the linearisation), channel r % CP
        constexpr int RL = ROWS / 32;
        int64_t roff[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int r = lane + 32 * q, nb = r / CP, ch = r % CP;
            roff[q] = ((int64_t)c * nx * ny + (nb >> 1) * nx + (nb & 1)) * CP + ch;
        }
        // one sweep over the sorted rows: column sums per run, and at the last
        // row of each run one atomic per (node, channel) (the run tests are
        // warp-uniform; each sum adds the run's rows in order)
        T acc[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) acc[q] = (T)0;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            if (jj >= nv) break;
#pragma unroll
            for (int q = 0; q < RL; ++q) acc[q] += tile[jj * RS + lane + 32 * q];
            if (jj == nv - 1 || ((heads >> (jj + 1)) & 1u)) {
                T* base = rho + (int64_t)__shfl_sync(FULL, cell, jj) * CP;
#pragma unroll
                for (int q = 0; q < RL; ++q) {
                    if ((lane + 32 * q) % CP < C) atomicAdd(base + roff[q], acc[q]);
                    acc[q] = (T)0;
                }
            }
        }
    }
    if (sb.key) {
        base = __shfl_sync(FULL, base, start & 31);
        if (sv) sb.rank[ps] = base + lane - start;
    }
    if (bad) atomicOr(err, bad);
}

template <typename T, int C, int CP, int WARPS, bool QS>
static __global__ void __launch_bounds__(WARPS * 32, dep_min_blocks<T, CP>()) deposit_tile_kernel(const T* __restrict__ state, int64_t N,
                                                                           const GeomDev* __restrict__ geom, int nx,
                                                                           int ny, int nz, T qm, T* __restrict__ rho,
                                                                           int* __restrict__ err, const SortBuf sb,
                                                                           int qslot, T qmd) {
    deposit_tile_body<T, C, CP, WARPS, QS>(state, N, geom, nx, ny, nz, qm, rho, err, sb, (int)blockIdx.x, qslot, qmd);
}

// ------------------------------------------------------------------ bounded-wait probe

// One thread polls an mbarrier that no one arrives on, `polls` times, and
// records how many polls failed: the device time of a wait that runs out.
static __global__ void wait_probe_kernel(int polls, int* failed) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    int f = 0;
    for (int it = 0; it < polls; ++it)
        if (!mbar_try_wait(&bar, 0u)) ++f;
    *failed = f;
}

}  // namespace adpic
