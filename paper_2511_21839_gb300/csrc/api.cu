// Host runtime behind the C ABI of include/ad_pic.h: handle and device memory,
// per-kick dual map coefficients (host FP64 dual arithmetic, Sec. 2 Eqs. 1-4
// applied to the quadrupole maps of Sec. 4), the split-step sequence of one
// run (Sec. 4, Eq. "map"), CUDA-graph capture and replay, per-kernel event
// timing, and the stage entry points used by the parity tests.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "ad_pic.h"
#include "common.cuh"
#include "handle.h"
#include "hostdual.h"

using namespace adpic;
using namespace adpic_host;

namespace {

// CODATA 2018
constexpr double kC = 299792458.0;
constexpr double kQE = 1.602176634e-19;

const char* kClassNames[kClasses] = {"push", "boundary", "deposit", "green", "fft", "field", "geometry", "misc"};
enum { K_PUSH = 0, K_BOUNDARY, K_DEPOSIT, K_GREEN, K_FFT, K_FIELD, K_GEOM, K_MISC };

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

}  // namespace



namespace {

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            std::fprintf(stderr, "ad_pic: %s failed: %s\n", #call, cudaGetErrorString(e_));   \
            return AD_PIC_ERR_CUDA;                                                            \
        }                                                                                      \
    } while (0)

// Host-side fault injection for the failure-handling tests (no GPU fault is
// ever made): ADPIC_FAULT=alloc:K makes every device allocation of a handle
// after its first K fail as if cudaMalloc had run out of memory;
// ADPIC_FAULT=launch makes ad_pic_run's launch report a failed launch.
int fault_alloc_after() {
    const char* f = std::getenv("ADPIC_FAULT");
    if (!f || std::strncmp(f, "alloc", 5) != 0) return -1;
    return f[5] == ':' ? std::atoi(f + 6) : 0;
}
bool fault_launch() {
    const char* f = std::getenv("ADPIC_FAULT");
    return f && std::strcmp(f, "launch") == 0;
}

// FP32 records [6 N][C] -> [6 N][CP] (padding channels zero)
__global__ void pad_records_f32_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t rows, int C,
                                       int CP) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows * CP) return;
    const int64_t r = t / CP;
    const int k = (int)(t % CP);
    dst[t] = k < C ? src[r * C + k] : 0.0f;
}
void pad_records_f32(const float* src, float* dst, int64_t N, int C, int CP, cudaStream_t s) {
    const int64_t rows = 6 * N;
    pad_records_f32_kernel<<<(unsigned)((rows * CP + 255) / 256), 256, 0, s>>>(src, dst, rows, C, CP);
}

int dalloc(ad_pic* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    const int after = fault_alloc_after();
    if (after >= 0 && (int)h->allocs.size() >= after) { *p = nullptr; return AD_PIC_ERR_OOM; }
    if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; cudaGetLastError(); return AD_PIC_ERR_OOM; }
    h->allocs.push_back(*p);
    return AD_PIC_OK;
}

void free_graphs(ad_pic* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

// event timing around the launches of the selected kernel classes
void tbegin(ad_pic* h, int cls, bool capturing, cudaStream_t st = nullptr) {
    if (!((h->tmask >> cls) & 1u)) return;
    if (!st) st = h->stream;
    while ((int)h->events.size() < h->ev_used + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->events.push_back(e);
    }
    if ((int)h->ev_class.size() < (h->ev_used + 2) / 2) h->ev_class.resize((h->ev_used + 2) / 2);
    h->ev_class[h->ev_used / 2] = cls;
    if (capturing) cudaEventRecordWithFlags(h->events[h->ev_used], st, cudaEventRecordExternal);
    else cudaEventRecord(h->events[h->ev_used], st);
}
void tend(ad_pic* h, int cls, bool capturing, cudaStream_t st = nullptr) {
    if (!((h->tmask >> cls) & 1u)) return;
    if (!st) st = h->stream;
    if (capturing) cudaEventRecordWithFlags(h->events[h->ev_used + 1], st, cudaEventRecordExternal);
    else cudaEventRecord(h->events[h->ev_used + 1], st);
    h->ev_used += 2;
}
void tcollect(ad_pic* h, int pairs) {
    for (int j = 0; j < pairs; ++j) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->events[2 * j], h->events[2 * j + 1]) == cudaSuccess) {
            h->tms[h->ev_class[j]] += ms;
            h->tcount[h->ev_class[j]] += 1;
        }
    }
    cudaGetLastError();
}

// ------------------------------------------------------------------ typed implementation

template <typename T, int C, int CP>
struct Impl {
    using M = MapCoef<T, CP>;
    using K = KickCoef<T, CP>;

    static T* buf(ad_pic* h, int b) { return (T*)(b ? h->state2 : h->state); }
    static T* st(ad_pic* h) { return buf(h, h->cur); }
    static SortBuf sortbuf(ad_pic* h, int from) {
        SortBuf sb;
        sb.key = h->key;
        sb.rank = h->rank;
        sb.hist = h->cellcount;
        sb.offs = h->offs;
        sb.ids_in = h->ids[from];
        sb.ids_out = h->ids[1 - from];
        sb.dst = h->dst;
        return sb;
    }
    // gather + kick + map A from buffer `from` into the other one, in cell-sorted order
    static void push(ad_pic* h, int& from, const MapCoef<T, CP>& A, const KickCoef<T, CP>& K, bool track) {
        launch_push<T, C, CP>(buf(h, from), buf(h, 1 - from), h->N, (const T*)h->E, h->geom, h->nx, h->ny, h->nz, A,
                              K, track, (Ord<T>*)h->mm, h->err, sortbuf(h, from), track ? gfuse(h) : no_fuse(),
                              h->wait_polls, h->stream);
        from = 1 - from;
    }

    static M to_map(const HMap& a) {
        M r;
        for (int p = 0; p < 3; ++p)
            for (int e = 0; e < 4; ++e)
                for (int k = 0; k < CP; ++k) r.m[p][e][k] = (T)a.m[p][e].v[k];
        return r;
    }
    static M identity() {
        HMap I;
        for (int p = 0; p < 3; ++p) { I.m[p][0] = hc(1); I.m[p][1] = hc(0); I.m[p][2] = hc(0); I.m[p][3] = hc(1); }
        return to_map(I);
    }

    // The reference-particle constants as host duals of the kinetic energy E
    // (slot eslot, Sec. 4: beam parameters as AD variables): gamma0 = 1 + E/m,
    // beta0 gamma0 = sqrt(gamma0^2 - 1), p0 = beta0 gamma0 m c, B rho = p0/q,
    // v0 = c beta0 gamma0 / gamma0, kappa_perp = q/(gamma0 p0 v0), kappa_z =
    // q/(p0 v0). The value parts are the handle's constants; without an energy
    // slot the derivative parts are zero.
    struct EConst {
        HD g0, g2, bg, brho, kperp, kz;
    };
    static EConst energy_consts(const ad_pic* h) {
        EConst e;
        if (h->eslot >= 0) {
            const double mass_kg = h->mass_eV * kQE / (kC * kC);
            const HD E = hvar((h->gamma0 - 1.0) * h->mass_eV, h->eslot);
            e.g0 = hadd(hc(1.0), hmul(E, hc(1.0 / h->mass_eV)));
            e.g2 = hmul(e.g0, e.g0);
            e.bg = hsqrt(hadd(e.g2, hc(-1.0)));
            const HD p0 = hmul(e.bg, hc(mass_kg * kC));
            e.brho = hdiv(p0, hc(h->q));
            const HD v0 = hmul(hdiv(e.bg, e.g0), hc(kC));
            e.kperp = hdiv(hc(h->q), hmul(hmul(e.g0, p0), v0));
            e.kz = hdiv(hc(h->q), hmul(p0, v0));
        } else {
            e.g0 = e.g2 = e.bg = e.brho = e.kperp = e.kz = hc(0.0);
        }
        e.g0.v[0] = h->gamma0;
        e.g2.v[0] = h->gamma0 * h->gamma0;
        e.bg.v[0] = h->beta0 * h->gamma0;
        e.brho.v[0] = h->brho;
        e.kperp.v[0] = h->kperp;
        e.kz.v[0] = h->kz;
        return e;
    }

    // per-kick dual coefficients of one period
    static void build_coef(ad_pic* h) {
        const EConst ec = energy_consts(h);
        const ad_pic_lattice& L = h->lat;
        const int len_param[5] = {0, 1, 3, 4, 6};
        const bool use_line = !h->line.empty();
        const int n_elem = use_line ? (int)h->line.size() : 5;
        auto kicks_of = [&](int e) { return use_line ? h->line_kicks[e] : L.kicks[e]; };
        int kpp = 0;
        for (int e = 0; e < n_elem; ++e) kpp += kicks_of(e);
        h->kpp = kpp;
        std::vector<HMap> halfm(kpp);
        std::vector<K> kc(kpp);
        int s = 0;
        for (int e = 0; e < n_elem; ++e) {
            HD Le = use_line ? hvar(h->line[e].L, h->line[e].slot_L) : hvar(L.L[e], L.deriv_slot[len_param[e]]);
            HD tau = hdiv(Le, hc((double)kicks_of(e)));      // D tau = D L / n (Sec. 4)
            HD t = hmul(tau, hc(0.5));
            HD kx = hc(0.0), ky = hc(0.0);
            if (use_line) {
                if (h->line[e].type == AD_PIC_QUAD) {        // normalised strength k, a dual of its own
                    kx = hvar(h->line[e].k, h->line[e].slot_k);
                    ky = hneg(kx);
                }
            } else if (e == 1 || e == 3) {
                const int gi = e == 1 ? 0 : 1;
                HD g = hvar(L.g[gi], L.deriv_slot[e == 1 ? 2 : 5]);
                kx = hdiv(g, ec.brho);                       // k = q g / p0 (B rho dual in the energy)
                ky = hneg(kx);
            }
            HMap m;
            plane_map(kx, t, m.m[0]);
            plane_map(ky, t, m.m[1]);
            m.m[2][0] = hc(1.0);
            m.m[2][1] = hdiv(t, ec.g2);                   // z += t delta / gamma0^2
            m.m[2][2] = hc(0.0);
            m.m[2][3] = hc(1.0);
            HD ap = hmul(ec.kperp, tau), az = hmul(ec.kz, tau);
            K kk;
            for (int k = 0; k < CP; ++k) { kk.a[0][k] = (T)ap.v[k]; kk.a[1][k] = (T)ap.v[k]; kk.a[2][k] = (T)az.v[k]; }
            for (int j = 0; j < kicks_of(e); ++j, ++s) { halfm[s] = m; kc[s] = kk; }
        }
        h->half.resize(sizeof(M) * kpp);
        h->comp.resize(sizeof(M) * kpp);
        h->kcoef.resize(sizeof(K) * kpp);
        for (int i = 0; i < kpp; ++i) {
            M a = to_map(halfm[i]);
            M c = to_map(compose(halfm[(i + 1) % kpp], halfm[i]));
            std::memcpy(h->half.data() + sizeof(M) * i, &a, sizeof(M));
            std::memcpy(h->comp.data() + sizeof(M) * i, &c, sizeof(M));
            std::memcpy(h->kcoef.data() + sizeof(K) * i, &kc[i], sizeof(K));
        }
        h->coef_dirty = false;
    }
    static const M& half(ad_pic* h, int64_t g) { return ((const M*)h->half.data())[g % h->kpp]; }
    static const M& comp(ad_pic* h, int64_t g) { return ((const M*)h->comp.data())[g % h->kpp]; }
    static const K& kick(ad_pic* h, int64_t g) { return ((const K*)h->kcoef.data())[g % h->kpp]; }

    static FFTDims dims(ad_pic* h) {
        FFTDims d;
        d.nx = h->nx; d.ny = h->ny; d.nz = h->nz;
        d.Mx = 2 * h->nx; d.My = 2 * h->ny; d.Mz = 2 * h->nz;
        d.lx = ilog2(d.Mx); d.ly = ilog2(d.My); d.lz = ilog2(d.Mz);
        d.C = C; d.CP = CP; d.npair = C / 2;
        d.norm = 1.0 / ((double)d.Mx * d.My * d.Mz);
        return d;
    }

    // the fused geometry step for the kernel that produces the extrema
    static GeomFuse gfuse(ad_pic* h) {
        GeomFuse f;
        f.count = h->gcount;
        f.nx = h->nx; f.ny = h->ny; f.nz = h->nz; f.CP = CP;
        f.gamma0 = h->gamma0;
        f.g = h->geom;
        f.chmax = h->chmax;
        return f;
    }
    static GeomFuse no_fuse() {
        GeomFuse f{};
        f.count = nullptr;
        return f;
    }

    // The kinetic energy as a dual input (eslot): the spectrum of dG/dE after
    // the Green's function on stream s, and the extra convolution (dG/dE) *
    // rho_0 added to the energy channel of phi. rho_0 was copied into the
    // two-channel records rho_e before the main convolution cleared rho; the
    // main convolution has waited for the spectra.
    static void green_energy(ad_pic* h, cudaStream_t s) {
        launch_green_energy<T>(h->geom, h->nx, h->ny, h->nz, h->corner, h->corner_e, (T*)h->G, (T*)h->Gtmp,
                               (T*)h->Ghat_e, (const T*)h->dct[0], (const T*)h->dct[1], (const T*)h->dct[2],
                               fft_slab_path<T>(dims(h)) ? 1 : 0, 1.0 / h->mass_eV, s);
    }
    static void energy_term(ad_pic* h, cudaStream_t s) {
        const int64_t nodes = (int64_t)h->nx * h->ny * h->nz;
        FFTDims de = dims(h);
        de.C = 2;
        de.CP = 2;
        de.npair = 1;
        launch_fft_conv<T>((T*)h->rho_e, (V2<T>*)h->X1, (V2<T>*)h->X2, (const T*)h->Ghat_e, (T*)h->phi_e, de,
                           (const V2<T>*)h->tw[0], (const V2<T>*)h->tw[1], (const V2<T>*)h->tw[2],
                           (const Ord<T>*)h->chmax, s);
        launch_energy_add<T>((const T*)h->phi_e, nodes, (T*)h->phi, CP, h->eslot + 1, s);
    }

    // deposit -> Green -> convolution -> field for the current state. The grid
    // geometry was derived by the last block of the kernel before (the push
    // that tracked the extrema, or the half map at a run or period start).
    // The convolution leaves rho zero for the next deposit.
    static void enqueue_field(ad_pic* h, int from, bool cap) {
        cudaStream_t s = h->stream;
        const int64_t nodes = (int64_t)h->nx * h->ny * h->nz;
        // Green's function on the side stream (it needs only the geometry)
        cudaEventRecord(h->ev_fork, s);
        cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        tbegin(h, K_GREEN, cap, h->side);
        launch_green<T>(h->geom, h->nx, h->ny, h->nz, sizeof(T) == 8, h->corner, (T*)h->G, (T*)h->Gtmp,
                        (T*)h->Ghat, (const T*)h->dct[0], (const T*)h->dct[1], (const T*)h->dct[2],
                        fft_slab_path<T>(dims(h)) ? 1 : 0, h->side);
        if (h->eslot >= 0) green_energy(h, h->side);
        tend(h, K_GREEN, cap, h->side);
        cudaEventRecord(h->ev_join, h->side);
        tbegin(h, K_DEPOSIT, cap);
        launch_deposit<T, C, CP>(buf(h, from), h->N, h->geom, h->nx, h->ny, h->nz, (T)h->qm, (T*)h->rho, h->err,
                                 sortbuf(h, from), h->qslot, s);
        tend(h, K_DEPOSIT, cap);
        // cell offsets for the push on the side stream, behind the Green's function
        cudaEventRecord(h->ev_dep, s);
        cudaStreamWaitEvent(h->side, h->ev_dep, 0);
        tbegin(h, K_MISC, cap, h->side);
        launch_scan(h->cellcount, h->offs, h->bsum, (int)nodes, h->side);
        launch_slots(h->key, h->rank, h->offs, h->dst, h->N, h->side);
        tend(h, K_MISC, cap, h->side);
        cudaEventRecord(h->ev_scan, h->side);
        tbegin(h, K_MISC, cap);
        launch_chmax<T>((const T*)h->rho, nodes, CP, (Ord<T>*)h->chmax, s);
        if (h->eslot >= 0) launch_energy_copy<T>((const T*)h->rho, CP, nodes, (T*)h->rho_e, s);
        tend(h, K_MISC, cap);
        tbegin(h, K_FFT, cap);
        FFTDims d = dims(h);
        // the forward x pass runs while the Green's spectrum is still being made
        launch_fft_conv<T>((T*)h->rho, (V2<T>*)h->X1, (V2<T>*)h->X2, (const T*)h->Ghat, (T*)h->phi, d,
                           (const V2<T>*)h->tw[0], (const V2<T>*)h->tw[1], (const V2<T>*)h->tw[2],
                           (const Ord<T>*)h->chmax, s, h->ev_join);
        if (h->eslot >= 0) energy_term(h, s);
        tend(h, K_FFT, cap);
        tbegin(h, K_FIELD, cap);
        launch_field<T>((const T*)h->phi, h->geom, h->nx, h->ny, h->nz, CP, (T*)h->E, s);
        if (h->eslot >= 0)
            launch_energy_field<T>((T*)h->E, nodes, CP, h->eslot + 1, 1.0 / (h->mass_eV * h->gamma0), s);
        tend(h, K_FIELD, cap);
        cudaStreamWaitEvent(s, h->ev_scan, 0);     // the push reads the cell offsets
    }

    static void record(ad_pic* h, int r, bool cap) {
        tbegin(h, K_MISC, cap);
        launch_moments_reduce(h->partial, boundary_blocks(), CP, h->N, h->records + (int64_t)r * 15 * CP, h->stream);
        tend(h, K_MISC, cap);
    }

    // kernels launched by one enqueue_field (deposit 1, scan 2, push slots 1,
    // chmax 1, Green's function 4: corners, cell averages with the first DCT
    // pass, two DCT passes; convolution 3 or 5, field 1); with the energy slot
    // also its Green's spectrum (4), the copy of rho_0, its convolution, the
    // add into phi and the E_z term
    static int field_launches(ad_pic* h) {
        const int conv = fft_conv_launches(fft_slab_path<T>(dims(h)));
        return 10 + conv + (h->eslot >= 0 ? 7 + conv : 0);
    }

    // the launch sequence of one run; returns the number of moment records
    // `from` is the buffer holding the particles at the start; each push moves
    // them to the other buffer in cell-sorted order
    static int enqueue_run(ad_pic* h, int64_t g0, int n, bool first, bool cap, int from) {
        cudaStream_t s = h->stream;
        const int nb = boundary_blocks();
        int nrec = 0;
        cudaMemsetAsync(h->err, 0, sizeof(int), s);
        if (n == 0) {
            tbegin(h, K_BOUNDARY, cap);
            launch_boundary<T, C, CP>(buf(h, from), h->N, identity(), false, true, h->partial, nb, (Ord<T>*)h->mm,
                                      no_fuse(), s);
            tend(h, K_BOUNDARY, cap);
            record(h, nrec++, cap);
            return nrec;
        }
        // opening half map M1(tau/2) of the first kick (+ initial moments)
        tbegin(h, K_BOUNDARY, cap);
        launch_boundary<T, C, CP>(buf(h, from), h->N, half(h, g0), true, first, h->partial, nb, (Ord<T>*)h->mm,
                                  gfuse(h), s);
        tend(h, K_BOUNDARY, cap);
        if (first) record(h, nrec++, cap);
        for (int i = 0; i < n; ++i) {
            const int64_t g = g0 + i;
            enqueue_field(h, from, cap);
            const bool last = i == n - 1;
            const bool pend = ((g + 1) % h->kpp) == 0;
            if (last || pend) {
                // M2(tau) then the closing M1(tau/2); moments at the period end,
                // then the next kick's opening M1(tau/2)
                tbegin(h, K_PUSH, cap);
                push(h, from, half(h, g), kick(h, g), false);
                tend(h, K_PUSH, cap);
                tbegin(h, K_BOUNDARY, cap);
                launch_boundary<T, C, CP>(buf(h, from), h->N, half(h, g + 1), !last, true, h->partial, nb,
                                          (Ord<T>*)h->mm, last ? no_fuse() : gfuse(h), s);
                tend(h, K_BOUNDARY, cap);
                record(h, nrec++, cap);
            } else {
                // M2(tau) then M1(tau/2) of this kick composed with M1(tau/2) of the next
                tbegin(h, K_PUSH, cap);
                push(h, from, comp(h, g), kick(h, g), true);
                tend(h, K_PUSH, cap);
            }
        }
        return nrec;
    }

    static int ensure_records(ad_pic* h, int n) {
        const int need = (h->first_record ? 1 : 0) + 1 + (int)(n / (h->kpp > 0 ? h->kpp : 1)) + 1;
        if (need > h->records_cap) {
            if (h->records) cudaFree(h->records);
            for (auto& p : h->allocs) if (p == h->records) p = nullptr;
            h->records = nullptr;
            int st_ = dalloc(h, (void**)&h->records, sizeof(double) * 15 * CP * need);
            if (st_) return st_;
            h->records_cap = need;
            free_graphs(h);
        }
        return AD_PIC_OK;
    }

    // append moment records [nrec][15][CP] to the history; advance counter and buffer parity
    static void finish(ad_pic* h, const double* rec, int nrec, int n) {
        for (int r = 0; r < nrec; ++r)
            for (int q = 0; q < 15; ++q)
                for (int k = 0; k < C; ++k) h->hist.push_back(rec[((size_t)r * 15 + q) * CP + k]);
        h->kick += n;
        h->first_record = false;
        if (n % 2) h->cur = 1 - h->cur;
    }

    static int prepare(ad_pic* h, int n, int* nrec) {
        if (h->coef_dirty) build_coef(h);
        int st_ = ensure_records(h, n);
        if (st_) return st_;
        *nrec = count_records(h, h->kick, n, h->first_record);
        return AD_PIC_OK;
    }

    static int run(ad_pic* h, int n) {
        if (h->coef_dirty) build_coef(h);
        const int64_t g0 = h->kick;
        const bool first = h->first_record;
        {
            int st_ = ensure_records(h, n);
            if (st_) return st_;
        }
        h->ev_used = 0;
        int nrec = 0;
        {
            // kernel launches of this run: opening boundary (+ reduce), per kick the field
            // kernels and the push, per moment record a boundary and a reduce
            const int nr = count_records(h, g0, n, first);
            int64_t l = 0;
            if (n == 0) l = 2;
            else l = 1 + (int64_t)n * (field_launches(h) + 1) + 2 * (int64_t)nr - (first ? 1 : 0);
            h->launches += l;
        }
        const int from = h->cur;
        if (h->use_graphs) {
            auto key = std::make_tuple((int)(g0 % h->kpp), n, first ? 1 : 0, h->tmask, from);
            auto it = h->graphs.find(key);
            if (it == h->graphs.end()) {
                cudaGraph_t graph;
                CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                nrec = enqueue_run(h, g0, n, first, true, from);
                CK(cudaStreamEndCapture(h->stream, &graph));
                cudaGraphExec_t ex;
                // captured launches keep their stream's priority
                CK(cudaGraphInstantiateWithFlags(&ex, graph, cudaGraphInstantiateFlagUseNodePriority));
                cudaGraphDestroy(graph);
                it = h->graphs.emplace(key, ex).first;
            } else {
                // replay: recompute the record count and event use without launching
                nrec = count_records(h, g0, n, first);
                h->ev_used = count_events(h, n, first, nrec);
            }
            CK(fault_launch() ? cudaErrorLaunchFailure : cudaGraphLaunch(it->second, h->stream));
        } else {
            if (fault_launch()) return AD_PIC_ERR_CUDA;
            nrec = enqueue_run(h, g0, n, first, false, from);
            CK(cudaGetLastError());
        }
        std::vector<double> rec((size_t)nrec * 15 * CP);
        int errw = 0;
        CK(cudaMemcpyAsync(rec.data(), h->records, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&errw, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (h->tmask) tcollect(h, h->ev_used / 2);
        finish(h, rec.data(), nrec, n);
        if (errw & kErrTimeout) {
            // a push gave up waiting for a state tile: some particles were not
            // pushed (nor their slots written), so the state must be set again
            h->particles_set = false;
            return AD_PIC_ERR_TIMEOUT;
        }
        if (errw & kErrNonfinite) return AD_PIC_ERR_NONFINITE;
        if (errw & kErrOutOfGrid) return AD_PIC_ERR_OUT_OF_GRID;
        return AD_PIC_OK;
    }

    static int count_records(ad_pic* h, int64_t g0, int n, bool first) {
        if (n == 0) return 1;
        int r = first ? 1 : 0;
        for (int i = 0; i < n; ++i) {
            const int64_t g = g0 + i;
            if (i == n - 1 || ((g + 1) % h->kpp) == 0) ++r;
        }
        return r;
    }
    static int count_events(ad_pic* h, int n, bool first, int nrec) {
        auto on = [&](int c) { return (int)((h->tmask >> c) & 1u); };
        if (n == 0) return 2 * (on(K_BOUNDARY) + on(K_MISC));
        int pend = nrec - (first ? 1 : 0);   // boundary+record pairs inside the loop
        int e = on(K_BOUNDARY) + (first ? on(K_MISC) : 0);
        e += n * (2 * on(K_MISC) + on(K_DEPOSIT) + on(K_GREEN) + on(K_FFT) + on(K_FIELD) + on(K_PUSH));
        // (the scan and chmax have one MISC event pair each)
        e += pend * (on(K_BOUNDARY) + on(K_MISC));
        return 2 * e;
    }

    // the energy term's buffers, once per handle
    static int alloc_energy(ad_pic* h) {
        if (h->Ghat_e) return AD_PIC_OK;
        const int64_t nodes = (int64_t)h->nx * h->ny * h->nz;
        const int64_t gnodes = (int64_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
        int r = 0;
        r |= dalloc(h, (void**)&h->corner_e, sizeof(double) * (h->nx + 2) * (h->ny + 2) * (h->nz + 2));
        r |= dalloc(h, &h->rho_e, sizeof(T) * nodes * 2);
        r |= dalloc(h, &h->phi_e, sizeof(T) * nodes * 2);
        if (!r) r |= dalloc(h, &h->Ghat_e, sizeof(T) * gnodes);    // last: its pointer marks success
        return r ? AD_PIC_ERR_OOM : AD_PIC_OK;
    }

    static int set_beam(ad_pic* h, const ad_pic_beam* b, const double* normals) {
        h->q = b->charge_e * kQE;
        const double mass_kg = b->mass_eV * kQE / (kC * kC);
        h->gamma0 = 1.0 + b->kinetic_eV / b->mass_eV;
        h->beta0 = std::sqrt(1.0 - 1.0 / (h->gamma0 * h->gamma0));
        h->p0 = h->gamma0 * h->beta0 * mass_kg * kC;
        h->brho = h->p0 / h->q;
        const double v0 = h->beta0 * kC;
        h->kperp = h->q / (h->gamma0 * h->p0 * v0);
        h->kz = h->q / (h->p0 * v0);
        h->qm = b->bunch_charge_C / (double)h->N;
        h->qslot = b->charge_deriv_slot;
        h->mass_eV = b->mass_eV;
        h->eslot = b->energy_deriv_slot;
        if (h->eslot >= 0 && alloc_energy(h)) {
            h->eslot = -1;
            return AD_PIC_ERR_OOM;
        }
        h->beam_set = true;
        h->coef_dirty = true;
        free_graphs(h);
        if (!normals) return AD_PIC_OK;
        const EConst ec = energy_consts(h);
        // per-plane dual coefficients u = a n1, p = b (n2 - alpha n1)
        std::vector<double> coef(3 * 3 * CP + 6, 0.0);
        const double bg = h->beta0 * h->gamma0;
        for (int pl = 0; pl < 3; ++pl) {
            const int sa = pl < 2 ? b->twiss_deriv_slot[3 * pl + 0] : -1;
            const int sb = pl < 2 ? b->twiss_deriv_slot[3 * pl + 1] : -1;
            const int se = pl < 2 ? b->twiss_deriv_slot[3 * pl + 2] : -1;
            HD al = hvar(b->alpha[pl], sa), be = hvar(b->beta[pl], sb);
            // geometric emittance eps_n / (beta0 gamma0), dual in the energy unless eps is a slot itself
            HD ep = (h->eslot >= 0 && se < 0) ? hdiv(hc(b->eps_n[pl]), ec.bg) : hvar(b->eps_n[pl] / bg, se);
            HD a = hsqrt(hmul(ep, be)), bb = hsqrt(hdiv(ep, be));
            for (int k = 0; k < CP; ++k) {
                coef[(pl * 3 + 0) * CP + k] = a.v[k];
                coef[(pl * 3 + 1) * CP + k] = bb.v[k];
                coef[(pl * 3 + 2) * CP + k] = al.v[k];
            }
        }
        for (int c = 0; c < 6; ++c) {
            double s = 0.0;
            for (int64_t i = 0; i < h->N; ++i) s += normals[(int64_t)c * h->N + i];
            coef[3 * 3 * CP + c] = s / (double)h->N;
        }
        double *nd = nullptr, *cd = nullptr;
        if (cudaMalloc(&nd, sizeof(double) * 6 * h->N) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_OOM; }
        if (cudaMalloc(&cd, sizeof(double) * coef.size()) != cudaSuccess) {
            cudaFree(nd);
            cudaGetLastError();
            return AD_PIC_ERR_OOM;
        }
        cudaError_t e1 = cudaMemcpyAsync(nd, normals, sizeof(double) * 6 * h->N, cudaMemcpyHostToDevice, h->stream);
        cudaError_t e2 = cudaMemcpyAsync(cd, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, h->stream);
        if (e1 == cudaSuccess && e2 == cudaSuccess) {
            launch_init<T, C, CP>(nd, h->N, cd, st(h), h->stream);
            launch_iota(h->ids[h->cur], h->N, h->stream);
        }
        cudaError_t e3 = cudaStreamSynchronize(h->stream);
        cudaFree(nd);
        cudaFree(cd);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || cudaGetLastError() != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        h->particles_set = true;
        h->kick = 0;
        h->first_record = true;
        h->hist.clear();
        return AD_PIC_OK;
    }

    static int staging(ad_pic* h, double** out) {
        if (!h->staging) {
            int r = dalloc(h, (void**)&h->staging, sizeof(double) * 6 * h->N * C);
            if (r) return r;
        }
        *out = h->staging;
        return AD_PIC_OK;
    }

    static int set_particles(ad_pic* h, const double* src) {
        double* tmp = nullptr;
        const size_t bytes = sizeof(double) * 6 * h->N * C;
        int r = staging(h, &tmp);
        if (r) return r;
        cudaError_t e1 = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, h->stream);
        if (e1 == cudaSuccess) {
            launch_convert_in<T, CP>(tmp, st(h), h->N, C, h->stream);
            launch_iota(h->ids[h->cur], h->N, h->stream);
        }
        cudaError_t e2 = cudaStreamSynchronize(h->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess || cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        h->particles_set = true;
        h->kick = 0;
        h->first_record = true;
        h->hist.clear();
        return AD_PIC_OK;
    }

    static int set_particles_f32(ad_pic* h, const float* src) {
        if (sizeof(T) != 4) return AD_PIC_ERR_UNSUPPORTED;
        const size_t bytes = sizeof(float) * 6 * h->N * C;
        cudaError_t e1;
        if (C == CP) {
            e1 = cudaMemcpyAsync(st(h), src, bytes, cudaMemcpyHostToDevice, h->stream);
        } else {
            double* tmp = nullptr;
            int r = staging(h, &tmp);                // holds 6 N C doubles: room for the floats
            if (r) return r;
            e1 = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, h->stream);
            if (e1 == cudaSuccess) pad_records_f32(reinterpret_cast<const float*>(tmp), (float*)st(h), h->N, C, CP,
                                                   h->stream);
        }
        if (e1 == cudaSuccess) launch_iota(h->ids[h->cur], h->N, h->stream);
        cudaError_t e2 = cudaStreamSynchronize(h->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess || cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        h->particles_set = true;
        h->kick = 0;
        h->first_record = true;
        h->hist.clear();
        return AD_PIC_OK;
    }

    // Asynchronous FP32 upload: the copy into the handle's prefetch buffer runs
    // on a copy stream of its own, after the previous commit has read that buffer
    static int prefetch_particles_f32(ad_pic* h, const float* src) {
        if (sizeof(T) != 4) return AD_PIC_ERR_UNSUPPORTED;
        const size_t bytes = sizeof(float) * 6 * h->N * C;
        if (!h->prefetch) {
            int r = dalloc(h, (void**)&h->prefetch, bytes);
            if (r) return r;
        }
        if (!h->copy) {
            if (cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_consumed, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(h->ev_consumed, h->stream) != cudaSuccess) {
                cudaGetLastError();
                return AD_PIC_ERR_CUDA;
            }
        }
        if (cudaStreamWaitEvent(h->copy, h->ev_consumed, 0) != cudaSuccess ||
            cudaMemcpyAsync(h->prefetch, src, bytes, cudaMemcpyHostToDevice, h->copy) != cudaSuccess ||
            cudaEventRecord(h->ev_copied, h->copy) != cudaSuccess) {
            cudaGetLastError();
            h->prefetched = false;
            return AD_PIC_ERR_CUDA;
        }
        h->prefetched = true;
        return AD_PIC_OK;
    }

    // the prefetched data becomes the particle state (as set_particles_f32),
    // ordered on the handle's stream after the copy; no host synchronisation
    static int commit_particles(ad_pic* h) {
        if (sizeof(T) != 4) return AD_PIC_ERR_UNSUPPORTED;
        if (!h->prefetched) return AD_PIC_ERR_STATE;
        const size_t bytes = sizeof(float) * 6 * h->N * C;
        cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_copied, 0);
        if (e == cudaSuccess) {
            if (C == CP)
                e = cudaMemcpyAsync(st(h), h->prefetch, bytes, cudaMemcpyDeviceToDevice, h->stream);
            else
                pad_records_f32(h->prefetch, (float*)st(h), h->N, C, CP, h->stream);
        }
        if (e == cudaSuccess) {
            launch_iota(h->ids[h->cur], h->N, h->stream);
            e = cudaEventRecord(h->ev_consumed, h->stream);
        }
        if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        h->prefetched = false;
        h->particles_set = true;
        h->kick = 0;
        h->first_record = true;
        h->hist.clear();
        return AD_PIC_OK;
    }

    static int get_particles(const ad_pic* hc_, double* dst) {
        ad_pic* h = const_cast<ad_pic*>(hc_);
        double* tmp = nullptr;
        const size_t bytes = sizeof(double) * 6 * h->N * C;
        int r = staging(h, &tmp);
        if (r) return r;
        launch_convert_out_perm<T, CP>(st(h), h->ids[h->cur], tmp, h->N, C, h->stream);
        cudaError_t e1 = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
        cudaError_t e2 = cudaStreamSynchronize(h->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess || cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        return AD_PIC_OK;
    }

    template <typename U>
    static void grid_out(const std::vector<U>& src, int comps, int64_t nodes, double* out) {
        // [node][comps][CP] -> [comps][C][node]
        for (int q = 0; q < comps; ++q)
            for (int k = 0; k < C; ++k)
                for (int64_t a = 0; a < nodes; ++a) out[((int64_t)q * C + k) * nodes + a] = (double)src[(a * comps + q) * CP + k];
    }

    static int stage(ad_pic* h, int which, int64_t kk, double* out) {
        if (h->coef_dirty) build_coef(h);
        cudaStream_t s = h->stream;
        const int64_t nodes = (int64_t)h->nx * h->ny * h->nz;
        CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
        launch_boundary<T, C, CP>(st(h), h->N, identity(), true, false, h->partial, boundary_blocks(),
                                  (Ord<T>*)h->mm, gfuse(h), s);     // with the geometry step
        if (which == 0) {
            GeomDev g;
            CK(cudaMemcpyAsync(&g, h->geom, sizeof(g), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int d = 0; d < 3; ++d) { out[d] = g.o[d]; out[3 + d] = g.h[d]; }
            return AD_PIC_OK;
        }
        // rho is zero between kicks (the convolution clears it); cleared here too
        CK(cudaMemsetAsync(h->rho, 0, sizeof(T) * nodes * CP, s));
        launch_deposit<T, C, CP>(st(h), h->N, h->geom, h->nx, h->ny, h->nz, (T)h->qm, (T*)h->rho, h->err,
                                 sortbuf(h, h->cur), h->qslot, s);
        launch_scan(h->cellcount, h->offs, h->bsum, (int)nodes, s);
        launch_slots(h->key, h->rank, h->offs, h->dst, h->N, s);
        std::vector<T> buf;
        if (which == 1) {
            buf.resize(nodes * CP);
            CK(cudaMemcpyAsync(buf.data(), h->rho, sizeof(T) * buf.size(), cudaMemcpyDeviceToHost, s));
            CK(cudaMemsetAsync(h->rho, 0, sizeof(T) * nodes * CP, s));   // no convolution follows
            CK(cudaStreamSynchronize(s));
            grid_out(buf, 1, nodes, out);
            return check_err(h);
        }
        launch_chmax<T>((const T*)h->rho, nodes, CP, (Ord<T>*)h->chmax, s);
        if (h->eslot >= 0) launch_energy_copy<T>((const T*)h->rho, CP, nodes, (T*)h->rho_e, s);
        launch_green<T>(h->geom, h->nx, h->ny, h->nz, sizeof(T) == 8, h->corner, (T*)h->G, (T*)h->Gtmp,
                        (T*)h->Ghat, (const T*)h->dct[0], (const T*)h->dct[1], (const T*)h->dct[2],
                        fft_slab_path<T>(dims(h)) ? 1 : 0, s);
        if (h->eslot >= 0) green_energy(h, s);
        FFTDims d = dims(h);
        launch_fft_conv<T>((T*)h->rho, (V2<T>*)h->X1, (V2<T>*)h->X2, (const T*)h->Ghat, (T*)h->phi, d,
                           (const V2<T>*)h->tw[0], (const V2<T>*)h->tw[1], (const V2<T>*)h->tw[2],
                           (const Ord<T>*)h->chmax, s);
        if (h->eslot >= 0) energy_term(h, s);
        if (which == 2) {
            buf.resize(nodes * CP);
            CK(cudaMemcpyAsync(buf.data(), h->phi, sizeof(T) * buf.size(), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            grid_out(buf, 1, nodes, out);
            return check_err(h);
        }
        launch_field<T>((const T*)h->phi, h->geom, h->nx, h->ny, h->nz, CP, (T*)h->E, s);
        if (h->eslot >= 0)
            launch_energy_field<T>((T*)h->E, nodes, CP, h->eslot + 1, 1.0 / (h->mass_eV * h->gamma0), s);
        if (which == 3) {
            buf.resize(nodes * 3 * CP);
            CK(cudaMemcpyAsync(buf.data(), h->E, sizeof(T) * buf.size(), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            grid_out(buf, 3, nodes, out);
            return check_err(h);
        }
        push(h, h->cur, identity(), kick(h, kk), false);
        CK(cudaStreamSynchronize(s));
        return check_err(h);
    }

    static int check_err(ad_pic* h) {
        int errw = 0;
        CK(cudaMemcpy(&errw, h->err, sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaGetLastError());
        if (errw & kErrTimeout) return AD_PIC_ERR_TIMEOUT;     // a bulk copy was not waited for
        if (errw & kErrNonfinite) return AD_PIC_ERR_NONFINITE;
        if (errw & kErrOutOfGrid) return AD_PIC_ERR_OUT_OF_GRID;
        return AD_PIC_OK;
    }

    // ---- checkpoint: the dual state of the handle's precision (with the
    // caller's particle index of every slot), the kick counter, the lattice,
    // the reference-particle constants and the moment history, so that a run
    // resumed from the file continues the same run
    struct FileHeader {
        char magic[8];
        uint32_t version, elem;
        int32_t prec, n_deriv, chans, chans_padded, nx, ny, nz, flags, first_record, qslot;
        int64_t N, kick, hist_len, n_line;
        double consts[8];
        ad_pic_lattice lat;
        int32_t eslot, pad;
        double mass_eV;
    };
    static constexpr size_t kChunk = (size_t)64 << 20;   // bytes staged on the host at a time

    static int save(ad_pic* h, const char* path) {
        if (!h->particles_set) return AD_PIC_ERR_STATE;
        FileHeader hd{};
        std::memcpy(hd.magic, "ADPICCK", 8);
        hd.version = 3;
        hd.elem = sizeof(T);
        hd.prec = h->prec; hd.n_deriv = h->P; hd.chans = C; hd.chans_padded = CP;
        hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz;
        hd.flags = (h->beam_set ? 1 : 0) | (h->lattice_set ? 2 : 0);
        hd.first_record = h->first_record ? 1 : 0;
        hd.qslot = h->qslot;
        hd.N = h->N; hd.kick = h->kick; hd.hist_len = (int64_t)h->hist.size(); hd.n_line = (int64_t)h->line.size();
        const double k[8] = {h->gamma0, h->beta0, h->p0, h->brho, h->kperp, h->kz, h->qm, h->q};
        std::memcpy(hd.consts, k, sizeof(k));
        hd.lat = h->lat;
        hd.eslot = h->eslot;
        hd.mass_eV = h->mass_eV;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return AD_PIC_ERR_CUDA;
        FILE* f = std::fopen(path, "wb");
        if (!f) return AD_PIC_ERR_IO;
        bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
        if (ok && !h->hist.empty()) ok = std::fwrite(h->hist.data(), sizeof(double), h->hist.size(), f) == h->hist.size();
        if (ok && !h->line.empty())
            ok = std::fwrite(h->line.data(), sizeof(ad_pic_element), h->line.size(), f) == h->line.size() &&
                 std::fwrite(h->line_kicks.data(), sizeof(int), h->line_kicks.size(), f) == h->line_kicks.size();
        std::vector<unsigned char> buf;
        auto dump = [&](const void* dev, size_t bytes) -> int {
            for (size_t o = 0; o < bytes && ok; o += kChunk) {
                const size_t n = bytes - o < kChunk ? bytes - o : kChunk;
                buf.resize(n);
                if (cudaMemcpy(buf.data(), (const unsigned char*)dev + o, n, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return AD_PIC_ERR_CUDA;
                ok = std::fwrite(buf.data(), 1, n, f) == n;
            }
            return AD_PIC_OK;
        };
        int st_ = dump(st(h), sizeof(T) * 6 * (size_t)h->N * CP);
        if (!st_) st_ = dump(h->ids[h->cur], sizeof(int) * (size_t)h->N);
        if (std::fclose(f) != 0) ok = false;
        if (st_) return st_;
        return ok ? AD_PIC_OK : AD_PIC_ERR_IO;
    }

    static int load(ad_pic* h, const char* path) {
        FILE* f = std::fopen(path, "rb");
        if (!f) return AD_PIC_ERR_IO;
        FileHeader hd{};
        int rc = AD_PIC_OK;
        if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "ADPICCK", 8) != 0 || hd.version != 3)
            rc = AD_PIC_ERR_IO;
        else if (hd.elem != sizeof(T) || hd.prec != h->prec || hd.n_deriv != h->P || hd.nx != h->nx || hd.ny != h->ny ||
                 hd.nz != h->nz || hd.N != h->N || hd.hist_len < 0 || hd.hist_len % (15 * C) != 0 || hd.n_line < 0 ||
                 hd.n_line > 100000)
            rc = AD_PIC_ERR_INVALID_ARG;      // a checkpoint of another configuration
        std::vector<double> hist;
        if (!rc) {
            hist.resize((size_t)hd.hist_len);
            if (!hist.empty() && std::fread(hist.data(), sizeof(double), hist.size(), f) != hist.size()) rc = AD_PIC_ERR_IO;
        }
        std::vector<ad_pic_element> line;
        std::vector<int> line_kicks;
        if (!rc && hd.n_line > 0) {
            line.resize((size_t)hd.n_line);
            line_kicks.resize((size_t)hd.n_line);
            if (std::fread(line.data(), sizeof(ad_pic_element), line.size(), f) != line.size() ||
                std::fread(line_kicks.data(), sizeof(int), line_kicks.size(), f) != line_kicks.size())
                rc = AD_PIC_ERR_IO;
        }
        std::vector<unsigned char> buf;
        auto fill = [&](void* dev, size_t bytes) {
            for (size_t o = 0; o < bytes && !rc; o += kChunk) {
                const size_t n = bytes - o < kChunk ? bytes - o : kChunk;
                buf.resize(n);
                if (std::fread(buf.data(), 1, n, f) != n) { rc = AD_PIC_ERR_IO; break; }
                if (cudaMemcpy((unsigned char*)dev + o, buf.data(), n, cudaMemcpyHostToDevice) != cudaSuccess)
                    rc = AD_PIC_ERR_CUDA;
            }
        };
        if (!rc) {
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = AD_PIC_ERR_CUDA;
        }
        if (!rc) fill(h->state, sizeof(T) * 6 * (size_t)h->N * CP);
        if (!rc) fill(h->ids[0], sizeof(int) * (size_t)h->N);
        std::fclose(f);
        if (rc) {
            // the device state may be partly overwritten: it must be set again
            h->particles_set = false;
            cudaGetLastError();
            return rc;
        }
        h->cur = 0;
        h->gamma0 = hd.consts[0]; h->beta0 = hd.consts[1]; h->p0 = hd.consts[2]; h->brho = hd.consts[3];
        h->kperp = hd.consts[4]; h->kz = hd.consts[5]; h->qm = hd.consts[6]; h->q = hd.consts[7];
        h->qslot = hd.qslot >= -1 && hd.qslot < h->P ? hd.qslot : -1;
        h->mass_eV = hd.mass_eV;
        h->eslot = hd.eslot >= 0 && hd.eslot < h->P && hd.mass_eV > 0 ? hd.eslot : -1;
        if (h->eslot >= 0 && alloc_energy(h)) {
            h->eslot = -1;
            h->particles_set = false;
            return AD_PIC_ERR_OOM;
        }
        h->beam_set = (hd.flags & 1) != 0;
        h->lattice_set = (hd.flags & 2) != 0;
        h->lat = hd.lat;
        h->line.swap(line);
        h->line_kicks.swap(line_kicks);
        h->particles_set = true;
        h->kick = hd.kick;
        h->first_record = hd.first_record != 0;
        h->hist.swap(hist);
        h->coef_dirty = true;
        free_graphs(h);
        return AD_PIC_OK;
    }

    static int allocate(ad_pic* h) {
        const int64_t nodes = (int64_t)h->nx * h->ny * h->nz;
        const int64_t gnodes = (int64_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
        const int npair = C / 2;
        const int Mx = 2 * h->nx, My = 2 * h->ny, Mz = 2 * h->nz;
        int r = 0;
        r |= dalloc(h, &h->state, sizeof(T) * 6 * h->N * CP);
        r |= dalloc(h, &h->state2, sizeof(T) * 6 * h->N * CP);
        // id and slot arrays carry 4 padding entries: the push copies their runs in 16-byte units
        r |= dalloc(h, (void**)&h->ids[0], sizeof(int) * (h->N + 4));
        r |= dalloc(h, (void**)&h->ids[1], sizeof(int) * (h->N + 4));
        r |= dalloc(h, (void**)&h->dst, sizeof(int) * (h->N + 4));
        r |= dalloc(h, (void**)&h->key, sizeof(int) * h->N);
        r |= dalloc(h, (void**)&h->rank, sizeof(int) * h->N);
        r |= dalloc(h, (void**)&h->cellcount, sizeof(int) * nodes);
        r |= dalloc(h, (void**)&h->offs, sizeof(int) * nodes);
        r |= dalloc(h, (void**)&h->bsum, sizeof(int) * (scan_blocks((int)nodes) + 1));
        r |= dalloc(h, &h->rho, sizeof(T) * nodes * CP);
        r |= dalloc(h, &h->phi, sizeof(T) * nodes * CP);
        r |= dalloc(h, &h->E, sizeof(T) * nodes * 3 * CP);
        r |= dalloc(h, &h->X1, sizeof(V2<T>) * npair * h->nz * h->ny * Mx);
        r |= dalloc(h, &h->X2, sizeof(V2<T>) * npair * h->nz * My * Mx);
        r |= dalloc(h, &h->G, sizeof(T) * gnodes);
        r |= dalloc(h, &h->Gtmp, sizeof(T) * gnodes);
        r |= dalloc(h, &h->Ghat, sizeof(T) * gnodes);
        r |= dalloc(h, (void**)&h->corner, sizeof(double) * (h->nx + 2) * (h->ny + 2) * (h->nz + 2));
        const int ns[3] = {h->nx, h->ny, h->nz};
        for (int d = 0; d < 3; ++d) r |= dalloc(h, &h->dct[d], sizeof(T) * (ns[d] + 1) * (ns[d] + 1));
        const int Ms[3] = {Mx, My, Mz};
        for (int d = 0; d < 3; ++d) r |= dalloc(h, &h->tw[d], sizeof(V2<T>) * Ms[d]);
        r |= dalloc(h, (void**)&h->geom, sizeof(GeomDev));
        r |= dalloc(h, &h->mm, sizeof(Ord<T>) * 6);
        r |= dalloc(h, &h->chmax, sizeof(Ord<T>) * CP);
        r |= dalloc(h, (void**)&h->err, sizeof(int));
        r |= dalloc(h, (void**)&h->gcount, sizeof(unsigned));
        r |= dalloc(h, (void**)&h->partial, sizeof(double) * boundary_blocks() * 15 * CP);
        if (r) return AD_PIC_ERR_OOM;
        CK(cudaMemsetAsync(h->state, 0, sizeof(T) * 6 * h->N * CP, h->stream));
        CK(cudaMemsetAsync(h->cellcount, 0, sizeof(int) * nodes, h->stream));
        CK(cudaMemsetAsync(h->rho, 0, sizeof(T) * nodes * CP, h->stream));
        CK(cudaMemsetAsync(h->gcount, 0, sizeof(unsigned), h->stream));
        launch_iota(h->ids[0], h->N, h->stream);
        launch_iota(h->ids[1], h->N, h->stream);
        CK(cudaMemsetAsync(h->E, 0, sizeof(T) * nodes * 3 * CP, h->stream));
        std::vector<Ord<T>> mm0 = {~(Ord<T>)0, ~(Ord<T>)0, ~(Ord<T>)0, 0, 0, 0};
        CK(cudaMemcpyAsync(h->mm, mm0.data(), sizeof(Ord<T>) * 6, cudaMemcpyHostToDevice, h->stream));
        // DCT-I matrices D[k][l] = w_l cos(pi l k / n) and FFT twiddles exp(-+ 2 pi i j / M)
        for (int d = 0; d < 3; ++d) {
            const int n = ns[d];
            std::vector<T> D((size_t)(n + 1) * (n + 1));
            for (int k = 0; k <= n; ++k)
                for (int l = 0; l <= n; ++l) {
                    const double w = (l == 0 || l == n) ? 1.0 : 2.0;
                    const long long m = ((long long)l * k) % (2LL * n);   // exact argument reduction
                    D[(size_t)k * (n + 1) + l] = (T)(w * std::cos(M_PI * (double)m / (double)n));
                }
            CK(cudaMemcpy(h->dct[d], D.data(), sizeof(T) * D.size(), cudaMemcpyHostToDevice));
            const int M = Ms[d];
            std::vector<V2<T>> f(M);
            for (int j = 0; j < M; ++j) {
                const double a = 2.0 * M_PI * (double)j / (double)M;
                f[j].x = (T)std::cos(a);
                f[j].y = (T)(-std::sin(a));
            }
            CK(cudaMemcpy(h->tw[d], f.data(), sizeof(V2<T>) * f.size(), cudaMemcpyHostToDevice));
        }
        setup_green<T>();
        setup_fft<T>();
        setup_deposit<T, C, CP>();
        setup_push<T, C, CP>();
        CK(cudaStreamSynchronize(h->stream));
        return AD_PIC_OK;
    }
};

// call Impl<T,C,CP>::fn for the handle's precision and derivative count
#define DISPATCH(h, expr)                                                      \
    do {                                                                       \
        if ((h)->prec == AD_PIC_FP64 && (h)->P == 7) { using I = Impl<double, 8, 8>; return expr; }   \
        if ((h)->prec == AD_PIC_FP64 && (h)->P == 13) { using I = Impl<double, 14, 16>; return expr; } \
        if ((h)->prec == AD_PIC_FP32_MIXED && (h)->P == 7) { using I = Impl<float, 8, 8>; return expr; } \
        if ((h)->prec == AD_PIC_FP32_MIXED && (h)->P == 13) { using I = Impl<float, 14, 16>; return expr; } \
        return AD_PIC_ERR_INVALID_ARG;                                         \
    } while (0)

}  // namespace

int adpic_prepare_run(ad_pic* h, int n_steps, int* n_records) { DISPATCH(h, I::prepare(h, n_steps, n_records)); }

void adpic_finish_run(ad_pic* h, const double* rec, int nrec, int n_steps) {
    auto f = [&]() -> int { DISPATCH(h, (I::finish(h, rec, nrec, n_steps), 0)); };
    f();
}

namespace {

// host dual emittance from one record [3][5][C]: centred moments, Eqs. for D eps
void emittance(const double* rec, int C, double* eps /*[3][C]*/) {
    for (int pl = 0; pl < 3; ++pl) {
        HD m[5];
        for (int q = 0; q < 5; ++q) {
            m[q] = hc(0.0);
            for (int k = 0; k < C; ++k) m[q].v[k] = rec[(pl * 5 + q) * C + k];
        }
        HD a = hadd(m[2], hneg(hmul(m[0], m[0])));
        HD b = hadd(m[3], hneg(hmul(m[0], m[1])));
        HD c = hadd(m[4], hneg(hmul(m[1], m[1])));
        HD e = hsqrt(hadd(hmul(a, c), hneg(hmul(b, b))));
        for (int k = 0; k < C; ++k) eps[pl * C + k] = e.v[k];
    }
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int ad_pic_create(const ad_pic_grid* grid, int64_t n_particles, int n_deriv, int precision, ad_pic** out) {
    if (!out) return AD_PIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || n_particles < 1 || n_particles > (int64_t)0x7fffffff) return AD_PIC_ERR_INVALID_ARG;
    if (n_deriv != 7 && n_deriv != 13) return AD_PIC_ERR_INVALID_ARG;
    if (precision != AD_PIC_FP64 && precision != AD_PIC_FP32_MIXED) return AD_PIC_ERR_INVALID_ARG;
    if (!pow2_in(grid->nx, 8, 128) || !pow2_in(grid->ny, 8, 128) || !pow2_in(grid->nz, 8, 128))
        return AD_PIC_ERR_INVALID_ARG;
    ad_pic* h = new (std::nothrow) ad_pic();
    if (!h) return AD_PIC_ERR_OOM;
    h->prec = precision;
    h->P = n_deriv;
    h->C = n_deriv + 1;
    h->CP = n_deriv == 7 ? 8 : 16;
    h->nx = grid->nx; h->ny = grid->ny; h->nz = grid->nz;
    h->N = n_particles;
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return AD_PIC_ERR_CUDA;
    }
    h->stream = h->own_stream;
    // the side stream (Green's function, then the cell offsets) at the highest
    // priority: the Green's spectrum is on the kick's critical path while its
    // kernels share the GPU with the deposit, so their blocks go first
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_dep, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_scan, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ad_pic_destroy(h);
        return AD_PIC_ERR_CUDA;
    }
    int st;
    auto alloc = [&]() -> int { DISPATCH(h, I::allocate(h)); };
    st = alloc();
    if (st) { ad_pic_destroy(h); return st; }
    *out = h;
    return AD_PIC_OK;
}

int ad_pic_set_beam(ad_pic* h, const ad_pic_beam* b, const double* normals) {
    if (!h || !b) return AD_PIC_ERR_INVALID_ARG;
    if (!(b->kinetic_eV > 0) || !(b->mass_eV > 0) || b->charge_e == 0 || !(b->bunch_charge_C >= 0))
        return AD_PIC_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(b->eps_n[d] > 0) || !(b->beta[d] > 0) || !std::isfinite(b->alpha[d])) return AD_PIC_ERR_INVALID_ARG;
    for (int j = 0; j < 6; ++j)
        if (b->twiss_deriv_slot[j] < -1 || b->twiss_deriv_slot[j] >= h->P) return AD_PIC_ERR_INVALID_ARG;
    if (b->charge_deriv_slot < -1 || b->charge_deriv_slot >= h->P) return AD_PIC_ERR_INVALID_ARG;
    if (b->energy_deriv_slot < -1 || b->energy_deriv_slot >= h->P ||
        (b->energy_deriv_slot >= 0 && b->energy_deriv_slot == b->charge_deriv_slot))
        return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::set_beam(h, b, normals));
}

int ad_pic_set_particles(ad_pic* h, const double* state) {
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::set_particles(h, state));
}

int ad_pic_set_particles_f32(ad_pic* h, const float* state) {
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::set_particles_f32(h, state));
}

int ad_pic_prefetch_particles_f32(ad_pic* h, const float* state) {
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::prefetch_particles_f32(h, state));
}

int ad_pic_commit_particles(ad_pic* h) {
    if (!h) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::commit_particles(h));
}

int ad_pic_get_particles(const ad_pic* h, double* state) {
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    if (!h->particles_set) return AD_PIC_ERR_STATE;
    DISPATCH(h, I::get_particles(h, state));
}

int ad_pic_set_lattice(ad_pic* h, const ad_pic_lattice* L) {
    if (!h || !L) return AD_PIC_ERR_INVALID_ARG;
    for (int e = 0; e < 5; ++e)
        if (!(L->L[e] > 0) || L->kicks[e] < 1 || L->kicks[e] > 100000) return AD_PIC_ERR_INVALID_ARG;
    if (!(L->g[0] != 0) || !(L->g[1] != 0) || !std::isfinite(L->g[0]) || !std::isfinite(L->g[1]))
        return AD_PIC_ERR_INVALID_ARG;
    for (int j = 0; j < 7; ++j)
        if (L->deriv_slot[j] < -1 || L->deriv_slot[j] >= h->P) return AD_PIC_ERR_INVALID_ARG;
    h->lat = *L;
    h->line.clear();
    h->line_kicks.clear();
    h->lattice_set = true;
    h->coef_dirty = true;
    free_graphs(h);
    return AD_PIC_OK;
}

int ad_pic_set_beamline(ad_pic* h, int n_elem, const ad_pic_element* elems, const int* kicks) {
    if (!h || n_elem < 1 || n_elem > 100000 || !elems || !kicks) return AD_PIC_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int e = 0; e < n_elem; ++e) {
        const ad_pic_element& x = elems[e];
        if (x.type != AD_PIC_DRIFT && x.type != AD_PIC_QUAD) return AD_PIC_ERR_INVALID_ARG;
        if (!(x.L > 0) || !std::isfinite(x.L) || (x.type == AD_PIC_QUAD && !std::isfinite(x.k)))
            return AD_PIC_ERR_INVALID_ARG;
        if (x.slot_L < -1 || x.slot_L >= h->P || x.slot_k < -1 || x.slot_k >= h->P) return AD_PIC_ERR_INVALID_ARG;
        if (kicks[e] < 1 || kicks[e] > 100000) return AD_PIC_ERR_INVALID_ARG;
        total += kicks[e];
    }
    if (total > 1000000) return AD_PIC_ERR_INVALID_ARG;
    h->line.assign(elems, elems + n_elem);
    h->line_kicks.assign(kicks, kicks + n_elem);
    h->lattice_set = true;
    h->coef_dirty = true;
    free_graphs(h);
    return AD_PIC_OK;
}

int ad_pic_run(ad_pic* h, int n_steps) {
    if (!h || n_steps < 0) return AD_PIC_ERR_INVALID_ARG;
    if (!h->beam_set || !h->lattice_set || !h->particles_set) return AD_PIC_ERR_STATE;
    DISPATCH(h, I::run(h, n_steps));
}

int ad_pic_moments_full(const ad_pic* h, double* mom) {
    if (!h || !mom) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    if (h->hist.size() < rs) return AD_PIC_ERR_STATE;
    std::memcpy(mom, h->hist.data() + h->hist.size() - rs, sizeof(double) * rs);
    return AD_PIC_OK;
}

int ad_pic_moments(const ad_pic* h, double* values, double* derivs) {
    if (!h || !values) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    if (h->hist.size() < rs) return AD_PIC_ERR_STATE;
    double eps[3 * kMaxCP];
    emittance(h->hist.data() + h->hist.size() - rs, h->C, eps);
    values[0] = eps[0];
    values[1] = eps[h->C];
    if (derivs)
        for (int k = 0; k < h->P; ++k) {
            derivs[k] = eps[1 + k];
            derivs[h->P + k] = eps[h->C + 1 + k];
        }
    return AD_PIC_OK;
}

int ad_pic_history(const ad_pic* h, double* hist, int max_records, int* n_records) {
    if (!h || !n_records || max_records < 0) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    const int n = (int)(h->hist.size() / rs);
    *n_records = n;
    if (hist) std::memcpy(hist, h->hist.data(), sizeof(double) * rs * (size_t)(n < max_records ? n : max_records));
    return AD_PIC_OK;
}

int ad_pic_set_stream(ad_pic* h, void* stream) {
    if (!h) return AD_PIC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_CUDA; }
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    free_graphs(h);
    return AD_PIC_OK;
}

int ad_pic_set_graphs(ad_pic* h, int enable) {
    if (!h) return AD_PIC_ERR_INVALID_ARG;
    h->use_graphs = enable != 0;
    if (!h->use_graphs) free_graphs(h);
    return AD_PIC_OK;
}

int ad_pic_set_timing(ad_pic* h, unsigned mask) {
    if (!h) return AD_PIC_ERR_INVALID_ARG;
    // graphs are keyed by the mask, so switching masks keeps the captured ones
    h->tmask = mask & ((1u << kClasses) - 1u);
    for (int c = 0; c < kClasses; ++c) { h->tms[c] = 0; h->tcount[c] = 0; }
    return AD_PIC_OK;
}

int ad_pic_timing(const ad_pic* h, double* ms, int64_t* launches, int n) {
    if (!h || n < 0) return AD_PIC_ERR_INVALID_ARG;
    for (int c = 0; c < n && c < kClasses; ++c) {
        if (ms) ms[c] = h->tms[c];
        if (launches) launches[c] = h->tcount[c];
    }
    return AD_PIC_OK;
}

const char* ad_pic_kernel_name(int cls) { return (cls >= 0 && cls < kClasses) ? kClassNames[cls] : "?"; }
int ad_pic_kernel_classes(void) { return kClasses; }

int ad_pic_stage(ad_pic* h, int stage, int64_t kick, double* out) {
    if (!h || stage < 0 || stage > 4 || (stage < 4 && !out) || kick < 0) return AD_PIC_ERR_INVALID_ARG;
    if (!h->beam_set || !h->particles_set || (stage == 4 && !h->lattice_set)) return AD_PIC_ERR_STATE;
    if (stage == 4 && h->coef_dirty && !h->lattice_set) return AD_PIC_ERR_STATE;
    if (!h->lattice_set) {
        // stages 0-3 need no lattice; use a placeholder period for the tables
        ad_pic_lattice L{};
        for (int e = 0; e < 5; ++e) { L.L[e] = 1.0; L.kicks[e] = 1; }
        L.g[0] = 1.0; L.g[1] = -1.0;
        for (int j = 0; j < 7; ++j) L.deriv_slot[j] = -1;
        h->lat = L;
        h->coef_dirty = true;
    }
    DISPATCH(h, I::stage(h, stage, kick, out));
}

int ad_pic_launches(const ad_pic* h, int64_t* n) {
    if (!h || !n) return AD_PIC_ERR_INVALID_ARG;
    *n = h->launches;
    return AD_PIC_OK;
}

int ad_pic_constants(const ad_pic* h, double* out) {
    if (!h || !out) return AD_PIC_ERR_INVALID_ARG;
    if (!h->beam_set) return AD_PIC_ERR_STATE;
    out[0] = h->gamma0; out[1] = h->beta0; out[2] = h->p0; out[3] = h->brho;
    out[4] = h->kperp; out[5] = h->kz; out[6] = h->qm; out[7] = h->q;
    return AD_PIC_OK;
}

int ad_pic_save(const ad_pic* h, const char* path) {
    if (!h || !path) return AD_PIC_ERR_INVALID_ARG;
    ad_pic* hm = const_cast<ad_pic*>(h);
    DISPATCH(hm, I::save(hm, path));
}

int ad_pic_load(ad_pic* h, const char* path) {
    if (!h || !path) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH(h, I::load(h, path));
}

int ad_pic_set_wait_limit(ad_pic* h, int polls) {
    if (!h) return AD_PIC_ERR_INVALID_ARG;
    h->wait_polls = polls < 0 ? -1 : polls;
    free_graphs(h);                  // the limit is a launch argument baked into the graphs
    return AD_PIC_OK;
}

int ad_pic_wait_probe(int polls, double* ms, int* failed) {
    if (polls < 1 || !ms || !failed) return AD_PIC_ERR_INVALID_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    int* d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = AD_PIC_OK;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_OOM; }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = AD_PIC_ERR_CUDA;
    if (!rc) {
        cudaEventRecord(e0, nullptr);
        if (launch_wait_probe(polls, d, nullptr)) rc = AD_PIC_ERR_CUDA;
        cudaEventRecord(e1, nullptr);
    }
    float t = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
                cudaMemcpy(failed, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = AD_PIC_ERR_CUDA;
    *ms = t;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (rc) cudaGetLastError();
    return rc;
}

void ad_pic_destroy(ad_pic* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->copy) cudaStreamSynchronize(h->copy);
    free_graphs(h);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_dep) cudaEventDestroy(h->ev_dep);
    if (h->ev_scan) cudaEventDestroy(h->ev_scan);
    if (h->copy) cudaStreamDestroy(h->copy);
    if (h->ev_copied) cudaEventDestroy(h->ev_copied);
    if (h->ev_consumed) cudaEventDestroy(h->ev_consumed);
    cudaGetLastError();
    delete h;
}

const char* ad_pic_strerror(int s) {
    switch (s) {
        case AD_PIC_OK: return "ok";
        case AD_PIC_ERR_INVALID_ARG: return "invalid argument";
        case AD_PIC_ERR_OOM: return "out of memory";
        case AD_PIC_ERR_CUDA: return "CUDA runtime error";
        case AD_PIC_ERR_STATE: return "call out of order";
        case AD_PIC_ERR_NONFINITE: return "non-finite particle coordinate";
        case AD_PIC_ERR_OUT_OF_GRID: return "particle outside the grid stencil";
        case AD_PIC_ERR_TIMEOUT: return "bounded device wait timed out";
        case AD_PIC_ERR_UNSUPPORTED: return "unsupported";
        case AD_PIC_ERR_IO: return "checkpoint file could not be read or written";
        case AD_PIC_ERR_UNSTABLE: return "cell has no periodic Twiss solution";
        default: return "unknown status";
    }
}

}  // extern "C"
