// Shared device types and launcher declarations of the GB300 dual-number PIC library.
//
// Storage (device):
//   state  T [6][N][CP]         coordinates (x, px, y, py, z, delta); channel 0 value,
//                               channels 1..C-1 derivatives, C..CP-1 zero padding so a
//                               particle's coordinate is 32 B (FP32, CP=8) / 64 B and
//                               moves in 32-byte pieces
//   rho    T [nz][ny][nx][CP]   node charges, channel-minor
//   phi    T [nz][ny][nx][CP]   potential
//   E      T [nz][ny][nx][3][CP] rest-frame field; boundary nodes stay zero
//   X1     V2 [npair][nz][ny][Mx]   spectrum after the x pass (M = 2n, zero padded)
//   X2     V2 [npair][nz][My][Mx]   after the y pass; the z pass works in place
//   Ghat   T [nz+1][ny+1][nx+1] real, even spectrum of the Green's function
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace adpic {

constexpr int kErrOutOfGrid = 1;
constexpr int kErrNonfinite = 2;
constexpr int kErrTimeout = 4;      // a bounded wait on a bulk copy gave up

template <typename T> struct V2T;
template <> struct V2T<float> { using type = float2; };
template <> struct V2T<double> { using type = double2; };
template <typename T> using V2 = typename V2T<T>::type;

// Lane-wise arithmetic on pairs. For FP32 one packed f32x2 instruction does
// both lanes (each lane rounds exactly as the scalar operation); FP64 pairs
// use two scalar operations.
#define ADPIC_F2_BINARY(name, op, fallback)                                                              \
    __device__ __forceinline__ float2 name(float2 a, float2 b) {                                         \
        float2 d;                                                                                        \
        asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n " op            \
            " rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                                                     \
            : "=f"(d.x), "=f"(d.y)                                                                       \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                   \
        return d;                                                                                        \
    }                                                                                                    \
    __device__ __forceinline__ double2 name(double2 a, double2 b) {                                      \
        double2 d;                                                                                       \
        d.x = a.x fallback b.x;                                                                          \
        d.y = a.y fallback b.y;                                                                          \
        return d;                                                                                        \
    }
ADPIC_F2_BINARY(v2_add, "add.rn.f32x2", +)
ADPIC_F2_BINARY(v2_sub, "sub.rn.f32x2", -)
ADPIC_F2_BINARY(v2_mul, "mul.rn.f32x2", *)
#undef ADPIC_F2_BINARY
__device__ __forceinline__ float2 v2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ double2 v2_fma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// ordered-integer encoding of floating point for atomicMin/atomicMax
template <typename T> struct OrdT;
template <> struct OrdT<float> { using type = unsigned int; };
template <> struct OrdT<double> { using type = unsigned long long; };
template <typename T> using Ord = typename OrdT<T>::type;

// ---------------------------------------------------------------- record access
// A record is the CP channels of one particle coordinate or one grid node:
// CP * sizeof(T) bytes, 16-byte aligned.
template <typename T, int CP>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&v)[CP]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q) {
            float4 f = reinterpret_cast<const float4*>(p)[q];
            v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < CP / 2; ++q) {
            double2 f = reinterpret_cast<const double2*>(p)[q];
            v[2 * q] = f.x; v[2 * q + 1] = f.y;
        }
    }
}

template <typename T, int CP>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&v)[CP]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < CP / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
    }
}

// Global accesses of whole records in 32-byte pieces (one request per piece):
// records are CP * sizeof(T) bytes with CP in {8, 16}, a multiple of 32, and
// every record starts on a 32-byte boundary of a cudaMalloc'ed array.
// ldg_v reads through the non-coherent path (data read-only in the kernel),
// ldr_v through the coherent one, stg_v stores. A translation unit that
// defines ADPIC_RECORD_ACCESS_16 before the include gets 16-byte pieces (the
// batched kernels: the assembler fails on their 32-byte form).
// L2 policy for data that is streamed through once (the particle state read by
// the deposit): its lines are evicted first, so the charge grid that the same
// kernel accumulates into stays resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
#ifdef ADPIC_RECORD_ACCESS_16
template <typename T, int CP>
__device__ __forceinline__ void ldg_v(const T* __restrict__ p, T (&v)[CP]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q) {
            float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
            v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < CP / 2; ++q) {
            double2 f = __ldg(reinterpret_cast<const double2*>(p) + q);
            v[2 * q] = f.x; v[2 * q + 1] = f.y;
        }
    }
}
template <typename T, int CP>
__device__ __forceinline__ void ldr_v(const T* p, T (&v)[CP]) { ldv<T, CP>(p, v); }
template <typename T, int CP>
__device__ __forceinline__ void stg_v(T* p, const T (&v)[CP]) { stv<T, CP>(p, v); }
template <typename T, int CP>
__device__ __forceinline__ void ldg_v_stream(const T* __restrict__ p, T (&v)[CP], uint64_t) { ldg_v<T, CP>(p, v); }
#else
template <typename T, int CP>
__device__ __forceinline__ void ldg_v(const T* __restrict__ p, T (&v)[CP]) {
    static_assert(CP * sizeof(T) % 32 == 0, "32-byte pieces");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 8; ++q)
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]), "=f"(v[8 * q + 4]),
                  "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
                : "l"(p + 8 * q));
    } else {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
            asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
                : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
                : "l"(p + 4 * q));
    }
}
template <typename T, int CP>
__device__ __forceinline__ void ldr_v(const T* p, T (&v)[CP]) {
    static_assert(CP * sizeof(T) % 32 == 0, "32-byte pieces");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 8; ++q)
            asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]), "=f"(v[8 * q + 4]),
                           "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
                         : "l"(p + 8 * q)
                         : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
                         : "l"(p + 4 * q)
                         : "memory");
    }
}
template <typename T, int CP>
__device__ __forceinline__ void stg_v(T* p, const T (&v)[CP]) {
    static_assert(CP * sizeof(T) % 32 == 0, "32-byte pieces");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 8; ++q)
            asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p + 8 * q), "f"(v[8 * q]),
                         "f"(v[8 * q + 1]), "f"(v[8 * q + 2]), "f"(v[8 * q + 3]), "f"(v[8 * q + 4]), "f"(v[8 * q + 5]),
                         "f"(v[8 * q + 6]), "f"(v[8 * q + 7])
                         : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
            asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 4 * q), "d"(v[4 * q]), "d"(v[4 * q + 1]),
                         "d"(v[4 * q + 2]), "d"(v[4 * q + 3])
                         : "memory");
    }
}
// a load with an L2 policy (l2_evict_first) for streamed records
template <typename T, int CP>
__device__ __forceinline__ void ldg_v_stream(const T* __restrict__ p, T (&v)[CP], uint64_t pol) {
    static_assert(CP * sizeof(T) % 32 == 0, "32-byte pieces");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < CP / 8; ++q)
            asm("ld.global.nc.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]), "=f"(v[8 * q + 4]),
                  "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
                : "l"(p + 8 * q), "l"(pol));
    } else {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
            asm("ld.global.nc.L2::cache_hint.v4.f64 {%0,%1,%2,%3}, [%4], %5;"
                : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
                : "l"(p + 4 * q), "l"(pol));
    }
}
#endif

// Grid geometry of one kick, computed on the device from the value-part extrema.
struct GeomDev {
    double o[3];    // origin (lab, m)
    double h[3];    // lab spacing (m)
    double hr[3];   // rest-frame spacing (hx, hy, gamma0 hz)
    float of[3], ihf[3];   // FP32 copies: origin and 1/h
    double ihd[3];         // 1/h
    float fdf[3];          // 1/(2 hr): central-difference factors (FP32 copy)
    double fdd[3];         // 1/(2 hr)
    int R[3];              // near-field box of the Green's function (cells per dimension)
};

// What a kernel that produces the value-part extrema needs to derive the grid
// geometry in its last block (count == nullptr: it does not).
struct GeomFuse {
    unsigned* count;        // finished blocks; zero between launches
    int nx, ny, nz, CP;
    double gamma0;
    GeomDev* g;
    void* chmax;            // Ord<T>[CP], reset with the extrema
};

// Dual 2x2 map per plane, entries (m11, m12, m21, m22).
template <typename T, int CP> struct MapCoef { T m[3][4][CP]; };
// Kick factors kappa_d * tau per field component (dual).
template <typename T, int CP> struct KickCoef { T a[3][CP]; };

struct FFTDims {
    int nx, ny, nz;
    int Mx, My, Mz;
    int lx, ly, lz;     // log2 of M
    int C, CP, npair;
    double norm;        // 1 / (Mx My Mz), set on the host (FP64 is slow on this part)
};

// ---------------------------------------------------------------- launchers
template <typename T, int C, int CP>
void launch_init(const double* normals_dev, int64_t N, const double* coef_dev, T* state, cudaStream_t s);
template <typename T, int CP>
void launch_convert_in(const double* src, T* dst, int64_t N, int C, cudaStream_t s);
template <typename T, int CP>
void launch_convert_out(const T* src, double* dst, int64_t N, int C, cudaStream_t s);

// Cell sort carried by the particle kernels: the deposit records each
// particle's cell (key) and its rank among the particles of that cell (hist
// counts them); the scan turns hist into exclusive offsets (offs) and clears
// hist; the push writes particle i to slot offs[key[i]] + rank[i] of the
// other state buffer and carries its id along (ids_out[slot] = ids_in[i]).
struct SortBuf {
    int* key;
    int* rank;
    int* hist;
    const int* offs;
    const int* ids_in;
    int* ids_out;
    // optional: the destination slot of every particle, offs[key[i]] + rank[i],
    // computed after the scan (nullptr: the push computes it itself). With it,
    // the persistent push copies each tile's slots and ids with its state.
    const int* dst;
};

// track: also reduce the value-part extrema of the new positions into mm; the
// last block then derives the next grid geometry when gf.count is set
// (launch_boundary likewise when it applies a map)
template <typename T, int C, int CP>
void launch_push(const T* state_in, T* state_out, int64_t N, const T* E, const GeomDev* geom, int nx, int ny, int nz,
                 const MapCoef<T, CP>& A, const KickCoef<T, CP>& K, bool track, Ord<T>* mm, int* err,
                 const SortBuf& sb, const GeomFuse& gf, int polls, cudaStream_t s);
// one thread polls an mbarrier nobody arrives on `polls` times (a bounded wait
// that runs out); *failed = the failed polls
int launch_wait_probe(int polls, int* failed, cudaStream_t s);
void launch_scan(int* hist, int* offs, int* bsum, int ncells, cudaStream_t s);
// dst[i] = offs[key[i]] + rank[i] for every particle
void launch_slots(const int* key, const int* rank, const int* offs, int* dst, int64_t N, cudaStream_t s);
int scan_blocks(int ncells);
void launch_iota(int* ids, int64_t N, cudaStream_t s);
template <typename T, int CP>
void launch_convert_out_perm(const T* src, const int* ids, double* dst, int64_t N, int C, cudaStream_t s);
template <typename T, int C, int CP>
void launch_boundary(T* state, int64_t N, const MapCoef<T, CP>& A, bool apply, bool mom, double* partial,
                     int nblocks, Ord<T>* mm, const GeomFuse& gf, cudaStream_t s);
int boundary_blocks();
template <typename T, int C, int CP>
void launch_deposit(const T* state, int64_t N, const GeomDev* geom, int nx, int ny, int nz, T qm, T* rho,
                    int* err, const SortBuf& sb, int qslot, cudaStream_t s);
template <typename T, int C, int CP>
void setup_deposit();
template <typename T, int C, int CP>
void setup_push();
void launch_moments_reduce(const double* partial, int nblocks, int CP, int64_t N, double* out, cudaStream_t s);

template <typename T>
void launch_chmax(const T* rho, int64_t nodes, int CP, Ord<T>* chmax, cudaStream_t s);
// Ghat order 0: [kz'][ky'][kx'] (x fastest); order 1: [kx'][kz'][ky'] (y fastest)
template <typename T>
void launch_green(const GeomDev* geom, int nx, int ny, int nz, bool exact, double* corner, T* G, T* Gtmp,
                  T* Ghat, const T* dct_x, const T* dct_y, const T* dct_z, int order, cudaStream_t s);
template <typename T>
void setup_green();
// the kinetic energy as a dual input: the spectrum of dG/dE (after launch_green
// on the same stream), and the extra convolution's input and output records
template <typename T>
void launch_green_energy(const GeomDev* geom, int nx, int ny, int nz, const double* corner, double* corner_e, T* G,
                         T* Gtmp, T* Ghat_e, const T* dct_x, const T* dct_y, const T* dct_z, int order,
                         double inv_mass_eV, cudaStream_t s);
template <typename T>
void launch_energy_copy(const T* rho, int CP, int64_t nodes, T* rho_e, cudaStream_t s);
template <typename T>
void launch_energy_add(const T* phi_e, int64_t nodes, T* phi, int CP, int ce, cudaStream_t s);
template <typename T>
void launch_energy_field(T* E, int64_t nodes, int CP, int ce, double r, cudaStream_t s);
template <typename T>
void setup_fft();
// twx/twy/twz: exp(-2 pi i j / M) for j < M of each axis (M = 2n)
// true when launch_fft_conv takes the three-launch slab path for these
// dimensions (it then expects Ghat in the [kx'][kz'][ky'] order, see launch_green)
template <typename T>
bool fft_slab_path(const FFTDims& d);
int fft_conv_launches(bool slab);
// rows per CTA of the slab path's x passes, and the dynamic shared memory of
// its kernels (which: 0 x pass, 1 (y, z) slab, 2 inverse x pass, else the
// largest), for callers that run their bodies elsewhere
template <typename T>
int fft_slab_yt(const FFTDims& d);
template <typename T>
size_t fft_slab_smem(const FFTDims& d, int which = -1);
// rho is read and left zero (ready for the next deposit). `spec`: an event
// the stream waits for after the forward x pass, before Ghat is first read
// (the spectrum made on another stream); null for none
template <typename T>
void launch_fft_conv(T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d,
                     const V2<T>* twx, const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s,
                     cudaEvent_t spec = nullptr);
template <typename T>
void launch_field(const T* phi, const GeomDev* geom, int nx, int ny, int nz, int CP, T* E, cudaStream_t s);

}  // namespace adpic
