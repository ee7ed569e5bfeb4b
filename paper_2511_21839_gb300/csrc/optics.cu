// Single-particle dual optics on the GPU (Sec. 3 of the paper): many
// beamlines of drifts and thick quadrupoles evaluated at once (Twiss
// transport, Eq. 5, and the periodic Twiss functions of a cell, with their
// derivatives w.r.t. element lengths and strengths), and batched
// element-by-element tracking of dual particles through a repeated beamline
// (the paper's 1000 turns x 100 FODO periods benchmark). Everything is FP64:
// Twiss functions of a strongly focusing cell and long-term tracking need it.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "ad_pic.h"

namespace {

// ------------------------------------------------------------------ device dual numbers
// A dual of CP channels: v[0] the value, v[k] the derivative w.r.t. slot k - 1.
template <int CP>
struct Dv {
    double v[CP];
};
template <int CP>
__device__ __forceinline__ Dv<CP> dconst(double x) {
    Dv<CP> r;
#pragma unroll
    for (int k = 0; k < CP; ++k) r.v[k] = 0.0;
    r.v[0] = x;
    return r;
}
template <int CP>
__device__ __forceinline__ Dv<CP> dvar(double x, int slot) {
    Dv<CP> r = dconst<CP>(x);
#pragma unroll
    for (int k = 1; k < CP; ++k)
        if (slot == k - 1) r.v[k] = 1.0;
    return r;
}
template <int CP>
__device__ __forceinline__ Dv<CP> dadd(const Dv<CP>& a, const Dv<CP>& b) {
    Dv<CP> r;
#pragma unroll
    for (int k = 0; k < CP; ++k) r.v[k] = a.v[k] + b.v[k];
    return r;
}
template <int CP>
__device__ __forceinline__ Dv<CP> dsub(const Dv<CP>& a, const Dv<CP>& b) {
    Dv<CP> r;
#pragma unroll
    for (int k = 0; k < CP; ++k) r.v[k] = a.v[k] - b.v[k];
    return r;
}
template <int CP>
__device__ __forceinline__ Dv<CP> dscale(double s, const Dv<CP>& a) {
    Dv<CP> r;
#pragma unroll
    for (int k = 0; k < CP; ++k) r.v[k] = s * a.v[k];
    return r;
}
// product rule (Eq. 2)
template <int CP>
__device__ __forceinline__ Dv<CP> dmul(const Dv<CP>& a, const Dv<CP>& b) {
    Dv<CP> r;
    r.v[0] = a.v[0] * b.v[0];
#pragma unroll
    for (int k = 1; k < CP; ++k) r.v[k] = fma(a.v[0], b.v[k], b.v[0] * a.v[k]);
    return r;
}
// quotient rule (Eq. 3)
template <int CP>
__device__ __forceinline__ Dv<CP> ddiv(const Dv<CP>& a, const Dv<CP>& b) {
    Dv<CP> r;
    const double q = a.v[0] / b.v[0], ib = 1.0 / b.v[0];
    r.v[0] = q;
#pragma unroll
    for (int k = 1; k < CP; ++k) r.v[k] = (a.v[k] - q * b.v[k]) * ib;
    return r;
}
// chain rule (Eq. 4) for a function with value h and derivative hp at a.v[0]
template <int CP>
__device__ __forceinline__ Dv<CP> dfn(const Dv<CP>& a, double h, double hp) {
    Dv<CP> r;
    r.v[0] = h;
#pragma unroll
    for (int k = 1; k < CP; ++k) r.v[k] = hp * a.v[k];
    return r;
}
template <int CP>
__device__ __forceinline__ Dv<CP> dsqrt(const Dv<CP>& a) {
    const double s = sqrt(a.v[0]);
    return dfn(a, s, 0.5 / s);
}

// dual 2x2 map of one plane over length L for strength kp (> 0 focusing,
// < 0 defocusing, 0 drift): the thick-lens matrix of Eq. "quadtr"
template <int CP>
__device__ void plane_map(const Dv<CP>& kp, const Dv<CP>& L, Dv<CP> (&m)[4]) {
    if (kp.v[0] > 0.0) {
        const Dv<CP> w = dsqrt(kp), th = dmul(w, L);
        double s, c;
        sincos(th.v[0], &s, &c);
        const Dv<CP> cs = dfn(th, c, -s), sn = dfn(th, s, c);
        m[0] = cs;
        m[1] = ddiv(sn, w);
        m[2] = dscale(-1.0, dmul(w, sn));
        m[3] = cs;
    } else if (kp.v[0] < 0.0) {
        const Dv<CP> w = dsqrt(dscale(-1.0, kp)), th = dmul(w, L);
        const double c = cosh(th.v[0]), s = sinh(th.v[0]);
        const Dv<CP> cs = dfn(th, c, s), sn = dfn(th, s, c);
        m[0] = cs;
        m[1] = ddiv(sn, w);
        m[2] = dmul(w, sn);
        m[3] = cs;
    } else {
        m[0] = dconst<CP>(1.0);
        m[1] = L;
        m[2] = dconst<CP>(0.0);
        m[3] = dconst<CP>(1.0);
    }
}

// acc <- e acc (e after acc along the beam)
template <int CP>
__device__ void mat_after(const Dv<CP> (&e)[4], Dv<CP> (&acc)[4]) {
    const Dv<CP> r0 = dadd(dmul(e[0], acc[0]), dmul(e[1], acc[2]));
    const Dv<CP> r1 = dadd(dmul(e[0], acc[1]), dmul(e[1], acc[3]));
    const Dv<CP> r2 = dadd(dmul(e[2], acc[0]), dmul(e[3], acc[2]));
    const Dv<CP> r3 = dadd(dmul(e[2], acc[1]), dmul(e[3], acc[3]));
    acc[0] = r0; acc[1] = r1; acc[2] = r2; acc[3] = r3;
}

template <int CP>
__device__ void element_plane_map(const ad_pic_element& e, int plane, Dv<CP> (&m)[4]) {
    const Dv<CP> L = dvar<CP>(e.L, e.slot_L);
    Dv<CP> k = e.type == AD_PIC_QUAD ? dvar<CP>(e.k, e.slot_k) : dconst<CP>(0.0);
    if (plane == 1) k = dscale(-1.0, k);
    plane_map(k, L, m);
}

// One thread per beamline instance. Per plane: the start Twiss functions
// (given, or the periodic solution of the first n_cell elements), then
// Eq. 5 through the remaining elements' matrix product.
template <int CP>
__global__ void __launch_bounds__(128) twiss_kernel(int n_inst, int n_elem, int n_cell,
                                                    const ad_pic_element* __restrict__ el,
                                                    const double* __restrict__ twiss0, int C, double* __restrict__ out,
                                                    int* __restrict__ status) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    const ad_pic_element* e = el + (size_t)inst * n_elem;
    int bad = 0;
    for (int pl = 0; pl < 2; ++pl) {
        Dv<CP> b0, a0;
        if (n_cell > 0) {
            Dv<CP> acc[4] = {dconst<CP>(1.0), dconst<CP>(0.0), dconst<CP>(0.0), dconst<CP>(1.0)};
            for (int i = 0; i < n_cell; ++i) {
                Dv<CP> m[4];
                element_plane_map<CP>(e[i], pl, m);
                mat_after(m, acc);
            }
            // cos mu = (m11 + m22) / 2; sin mu takes the sign of m12
            const Dv<CP> cs = dscale(0.5, dadd(acc[0], acc[3]));
            if (!(fabs(cs.v[0]) < 1.0)) bad = 1;
            Dv<CP> sn = dsqrt(dsub(dconst<CP>(1.0), dmul(cs, cs)));
            if (acc[1].v[0] < 0.0) sn = dscale(-1.0, sn);
            b0 = ddiv(acc[1], sn);
            a0 = ddiv(dscale(0.5, dsub(acc[0], acc[3])), sn);
        } else {
            b0 = dconst<CP>(twiss0[(size_t)inst * 4 + 2 * pl]);
            a0 = dconst<CP>(twiss0[(size_t)inst * 4 + 2 * pl + 1]);
        }
        Dv<CP> m[4] = {dconst<CP>(1.0), dconst<CP>(0.0), dconst<CP>(0.0), dconst<CP>(1.0)};
        for (int i = n_cell; i < n_elem; ++i) {
            Dv<CP> em[4];
            element_plane_map<CP>(e[i], pl, em);
            mat_after(em, m);
        }
        // Eq. 5 with gamma0 = (1 + alpha0^2) / beta0
        const Dv<CP> g0 = ddiv(dadd(dconst<CP>(1.0), dmul(a0, a0)), b0);
        const Dv<CP> beta = dadd(dsub(dmul(dmul(m[0], m[0]), b0), dscale(2.0, dmul(dmul(m[0], m[1]), a0))),
                                 dmul(dmul(m[1], m[1]), g0));
        const Dv<CP> alpha = dsub(dadd(dscale(-1.0, dmul(dmul(m[0], m[2]), b0)),
                                       dmul(dadd(dmul(m[0], m[3]), dmul(m[1], m[2])), a0)),
                                  dmul(dmul(m[1], m[3]), g0));
        double* o = out + (size_t)inst * 4 * C;
        for (int k = 0; k < C; ++k) {
            o[(2 * pl) * C + k] = beta.v[k];
            o[(2 * pl + 1) * C + k] = alpha.v[k];
        }
    }
    if (bad) atomicOr(status, 1);
}

// ------------------------------------------------------------------ tracking

// Per element and plane the dual map entries, stored as [4][KP] (value then
// the KP - 1 derivative channels, padded to a multiple of the chunk).
constexpr int kChunk = 8;     // derivative channels per thread

// One thread per (particle, chunk of kChunk derivative channels). Every
// thread carries the particle's values (x, px, y, py) and its chunk's
// derivatives, so the chunks of one particle never communicate: the map is
// linear, d(m x)/dp_k = m dx/dp_k + (dm/dp_k) x.
__global__ void __launch_bounds__(128) track_kernel(int64_t n_part, int n_chunks, int n_elem, int KP,
                                                    const double* __restrict__ maps, int64_t n_repeat,
                                                    const double* __restrict__ x0, double* __restrict__ out, int C) {
    extern __shared__ double sm[];             // [n_elem][2][4][KP]
    const int msize = n_elem * 2 * 4 * KP;
    for (int j = threadIdx.x; j < msize; j += blockDim.x) sm[j] = maps[j];
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_part * n_chunks) return;
    const int64_t p = t / n_chunks;
    const int ch = (int)(t - p * n_chunks);
    const int k0 = 1 + ch * kChunk;           // first derivative channel of this chunk
    double v[4], d[4][kChunk];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        v[c] = x0[p * 4 + c];
#pragma unroll
        for (int k = 0; k < kChunk; ++k) d[c][k] = 0.0;
    }
    for (int64_t r = 0; r < n_repeat; ++r) {
        for (int i = 0; i < n_elem; ++i) {
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                const double* m = sm + (size_t)(i * 2 + pl) * 4 * KP;
                const double x = v[2 * pl], px = v[2 * pl + 1];
                const double m11 = m[0], m12 = m[KP], m21 = m[2 * KP], m22 = m[3 * KP];
#pragma unroll
                for (int k = 0; k < kChunk; ++k) {
                    const double dx = d[2 * pl][k], dp = d[2 * pl + 1][k];
                    d[2 * pl][k] = fma(m11, dx, fma(m12, dp, fma(m[k0 + k], x, m[KP + k0 + k] * px)));
                    d[2 * pl + 1][k] = fma(m21, dx, fma(m22, dp, fma(m[2 * KP + k0 + k], x, m[3 * KP + k0 + k] * px)));
                }
                v[2 * pl] = fma(m11, x, m12 * px);
                v[2 * pl + 1] = fma(m21, x, m22 * px);
            }
        }
    }
    double* o = out + p * 4 * C;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (ch == 0) o[c * C] = v[c];
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
            if (k0 + k < C) o[c * C + k0 + k] = d[c][k];
    }
}

// ------------------------------------------------------------------ host side

// host dual numbers for the element maps of the tracking kernel (FP64, up to 33 channels)
constexpr int kMaxC = 33;
struct HDual {
    double v[kMaxC];
};
HDual hconst(double x) { HDual r{}; r.v[0] = x; return r; }
HDual hvar(double x, int slot) { HDual r = hconst(x); if (slot >= 0 && slot + 1 < kMaxC) r.v[slot + 1] = 1.0; return r; }
HDual hmul(const HDual& a, const HDual& b) {
    HDual r;
    r.v[0] = a.v[0] * b.v[0];
    for (int k = 1; k < kMaxC; ++k) r.v[k] = b.v[0] * a.v[k] + a.v[0] * b.v[k];
    return r;
}
HDual hdiv(const HDual& a, const HDual& b) {
    HDual r;
    r.v[0] = a.v[0] / b.v[0];
    for (int k = 1; k < kMaxC; ++k) r.v[k] = (a.v[k] * b.v[0] - b.v[k] * a.v[0]) / (b.v[0] * b.v[0]);
    return r;
}
HDual hfn(const HDual& a, double h, double hp) {
    HDual r;
    r.v[0] = h;
    for (int k = 1; k < kMaxC; ++k) r.v[k] = hp * a.v[k];
    return r;
}
HDual hneg(const HDual& a) { HDual r; for (int k = 0; k < kMaxC; ++k) r.v[k] = -a.v[k]; return r; }

void host_plane_map(const HDual& kp, const HDual& L, HDual (&m)[4]) {
    if (kp.v[0] > 0.0) {
        const double s0 = std::sqrt(kp.v[0]);
        const HDual w = hfn(kp, s0, 0.5 / s0), th = hmul(w, L);
        const HDual c = hfn(th, std::cos(th.v[0]), -std::sin(th.v[0])), s = hfn(th, std::sin(th.v[0]), std::cos(th.v[0]));
        m[0] = c; m[1] = hdiv(s, w); m[2] = hneg(hmul(w, s)); m[3] = c;
    } else if (kp.v[0] < 0.0) {
        const HDual nk = hneg(kp);
        const double s0 = std::sqrt(nk.v[0]);
        const HDual w = hfn(nk, s0, 0.5 / s0), th = hmul(w, L);
        const HDual c = hfn(th, std::cosh(th.v[0]), std::sinh(th.v[0])), s = hfn(th, std::sinh(th.v[0]), std::cosh(th.v[0]));
        m[0] = c; m[1] = hdiv(s, w); m[2] = hmul(w, s); m[3] = c;
    } else {
        m[0] = hconst(1.0); m[1] = L; m[2] = hconst(0.0); m[3] = hconst(1.0);
    }
}

bool valid_elements(int n_elem, const ad_pic_element* el, int n_deriv, size_t count) {
    for (size_t i = 0; i < count; ++i) {
        const ad_pic_element& e = el[i];
        if (e.type != AD_PIC_DRIFT && e.type != AD_PIC_QUAD) return false;
        if (!(e.L >= 0.0) || !std::isfinite(e.L) || (e.type == AD_PIC_QUAD && !std::isfinite(e.k))) return false;
        if (e.slot_L < -1 || e.slot_L >= n_deriv || e.slot_k < -1 || e.slot_k >= n_deriv) return false;
    }
    return n_elem >= 0;
}

template <typename F>
int with_device_buffers(size_t n, void** ptrs, const size_t* bytes, F&& body) {
    for (size_t i = 0; i < n; ++i) ptrs[i] = nullptr;
    int rc = AD_PIC_OK;
    for (size_t i = 0; i < n && !rc; ++i)
        if (cudaMalloc(&ptrs[i], bytes[i] ? bytes[i] : 16) != cudaSuccess) rc = AD_PIC_ERR_OOM;
    if (!rc) rc = body();
    for (size_t i = 0; i < n; ++i)
        if (ptrs[i]) cudaFree(ptrs[i]);
    if (rc) cudaGetLastError();
    return rc;
}

}  // namespace

extern "C" {

int ad_pic_twiss_batch(int n_inst, int n_elem, const ad_pic_element* elems, int n_deriv, int n_cell,
                       const double* twiss0, double* out) {
    if (n_inst < 1 || n_elem < 0 || n_elem > 4096 || !elems || !out || n_deriv < 0 || n_deriv > 15 || n_cell < 0 ||
        n_cell > n_elem || (n_cell == 0 && !twiss0))
        return AD_PIC_ERR_INVALID_ARG;
    if (!valid_elements(n_elem, elems, n_deriv, (size_t)n_inst * n_elem)) return AD_PIC_ERR_INVALID_ARG;
    if (n_cell == 0)
        for (int i = 0; i < n_inst; ++i)
            if (!(twiss0[4 * i] > 0.0) || !(twiss0[4 * i + 2] > 0.0)) return AD_PIC_ERR_INVALID_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    const int C = n_deriv + 1;
    void* d[4];
    const size_t bytes[4] = {sizeof(ad_pic_element) * (size_t)n_inst * n_elem,
                             n_cell == 0 ? sizeof(double) * 4 * (size_t)n_inst : 16,
                             sizeof(double) * 4 * (size_t)C * n_inst, sizeof(int)};
    return with_device_buffers(4, d, bytes, [&]() -> int {
        if (cudaMemcpy(d[0], elems, bytes[0], cudaMemcpyHostToDevice) != cudaSuccess) return AD_PIC_ERR_CUDA;
        if (n_cell == 0 && cudaMemcpy(d[1], twiss0, bytes[1], cudaMemcpyHostToDevice) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        if (cudaMemset(d[3], 0, sizeof(int)) != cudaSuccess) return AD_PIC_ERR_CUDA;
        const unsigned grid = (unsigned)((n_inst + 127) / 128);
        const ad_pic_element* e = (const ad_pic_element*)d[0];
        if (C <= 8)
            twiss_kernel<8><<<grid, 128>>>(n_inst, n_elem, n_cell, e, (const double*)d[1], C, (double*)d[2], (int*)d[3]);
        else
            twiss_kernel<16><<<grid, 128>>>(n_inst, n_elem, n_cell, e, (const double*)d[1], C, (double*)d[2], (int*)d[3]);
        if (cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        int st = 0;
        if (cudaMemcpy(out, d[2], bytes[2], cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&st, d[3], sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        return st ? AD_PIC_ERR_UNSTABLE : AD_PIC_OK;
    });
}

int ad_pic_track_batch(int64_t n_part, const double* x0, int n_elem, const ad_pic_element* elems, int n_deriv,
                       int64_t n_repeat, double* out, double* ms) {
    if (n_part < 1 || !x0 || !out || n_elem < 0 || !elems || n_deriv < 0 || n_deriv > 32 || n_repeat < 0)
        return AD_PIC_ERR_INVALID_ARG;
    if (!valid_elements(n_elem, elems, n_deriv, (size_t)n_elem)) return AD_PIC_ERR_INVALID_ARG;
    const int C = n_deriv + 1;
    const int n_chunks = n_deriv > 0 ? (n_deriv + kChunk - 1) / kChunk : 1;
    const int KP = 1 + n_chunks * kChunk;
    const size_t smem = sizeof(double) * (size_t)n_elem * 2 * 4 * KP;
    if (smem > 200 * 1024) return AD_PIC_ERR_UNSUPPORTED;       // the maps must fit in shared memory
    if (n_part > ((int64_t)1 << 40) / n_chunks) return AD_PIC_ERR_INVALID_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    // element maps (dual, host FP64), [n_elem][2][4][KP]
    std::vector<double> maps((size_t)n_elem * 2 * 4 * KP, 0.0);
    for (int i = 0; i < n_elem; ++i) {
        const ad_pic_element& e = elems[i];
        for (int pl = 0; pl < 2; ++pl) {
            HDual L = hvar(e.L, e.slot_L);
            HDual k = e.type == AD_PIC_QUAD ? hvar(e.k, e.slot_k) : hconst(0.0);
            if (pl == 1) k = hneg(k);
            HDual m[4];
            host_plane_map(k, L, m);
            for (int j = 0; j < 4; ++j)
                for (int c = 0; c < C; ++c) maps[(((size_t)i * 2 + pl) * 4 + j) * KP + c] = m[j].v[c];
        }
    }
    void* d[3];
    const size_t bytes[3] = {sizeof(double) * maps.size(), sizeof(double) * 4 * (size_t)n_part,
                             sizeof(double) * 4 * (size_t)C * n_part};
    return with_device_buffers(3, d, bytes, [&]() -> int {
        if (cudaMemcpy(d[0], maps.data(), bytes[0], cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d[1], x0, bytes[1], cudaMemcpyHostToDevice) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(track_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        const int64_t threads = n_part * n_chunks;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, nullptr);
        track_kernel<<<(unsigned)((threads + 127) / 128), 128, smem>>>(n_part, n_chunks, n_elem, KP,
                                                                         (const double*)d[0], n_repeat,
                                                                         (const double*)d[1], (double*)d[2], C);
        cudaEventRecord(e1, nullptr);
        int rc = cudaGetLastError() == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
        float t = 0.f;
        if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            rc = AD_PIC_ERR_CUDA;
        if (ms) *ms = t;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!rc && cudaMemcpy(out, d[2], bytes[2], cudaMemcpyDeviceToHost) != cudaSuccess) rc = AD_PIC_ERR_CUDA;
        return rc;
    });
}

}  // extern "C"
