// Batched runtime: many dual PIC instances (uneven particle counts, cubic
// grids of different sizes, P = 7, one lattice each) advanced together, as a
// sensitivity scan or an optimiser's line search needs.
//
// Every kernel body of the single-instance path takes an explicit block
// index, so one persistent cooperative kernel can walk, for each kick, the
// phases of the split step for all instances at once: within a phase the
// virtual blocks of every instance's jobs form one prefix-summed list that the
// resident blocks stride through; phases are separated by grid-wide
// barriers (cooperative launch, so every block is resident and no wait can
// stall on an absent block). The same phase code also runs as one ordinary
// launch per phase ("phased" mode). An autotuner times the persistent kernel
// at one and two blocks per SM against the phased launches on one kick of the
// actual batch and keeps the fastest. Runs are captured in CUDA graphs.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>
#include <string>
#include <mutex>

#include "ad_pic.h"
#define ADPIC_RECORD_ACCESS_16
#include "field_dev.cuh"
#include "fft_dev.cuh"
#include "handle.h"
#include "particles_dev.cuh"

namespace cg = cooperative_groups;
using namespace adpic;

namespace {

constexpr int kCP = 8;                  // P = 7

// Tile shapes of the jobs whose work split is free (the autotuner picks them):
// virtual blocks per instance of the moment pass, of the channel maxima and of
// the charge-grid clear, and 256-thread field blocks per virtual block.
struct Tiles {
    int bound_blocks = 8;
    int chmax_blocks = 4;
    int clear_blocks = 8;
    int field_per = 8;
};
constexpr int kTileChoices[4][4] = {{4, 8, 16, 32}, {2, 4, 8, 16}, {4, 8, 16, 32}, {2, 4, 8, 16}};

template <typename T>
struct Inst {
    int n, M;
    int64_t N;
    T qm;
    double gamma0;
    FFTDims d;
    int yt;             // rows per CTA of the slab x passes
    T* state[2];
    int* ids[2];
    int *key, *rank, *cellcount, *offs, *bsum;
    T *rho, *phi, *E;
    V2<T>*X1, *X2;
    T *G, *Gtmp, *Ghat;
    double* corner;
    const T* dct;
    const V2<T>* tw;
    GeomDev* geom;
    Ord<T>* mm;
    Ord<T>* chmax;
    int* err;
    double* partial;
    double* records;
    const MapCoef<T, kCP>* half;
    const MapCoef<T, kCP>* comp;
    const KickCoef<T, kCP>* kick;
    Tiles tiles;
};

enum Job {
    J_GEOM, J_CLEAR, J_DEPOSIT, J_CORNER, J_SCANSUM, J_CHMAX, J_CELL, J_SCANTOP, J_DCTX, J_SCANAPPLY, J_DCTY,
    J_DCTZ, J_FFTX, J_FFTYZ, J_FFTXI, J_FIELD, J_PUSH, J_BOUND, J_REDUCE, J_COUNT
};

// phases of one kick: the jobs of a phase depend only on earlier phases
enum Phase { PH_GEOM, PH_DEP, PH_2, PH_3, PH_4, PH_5, PH_FFTYZ, PH_FFTXI, PH_FIELD, PH_PUSH, PH_BOUND, PH_REDUCE,
             PH_COUNT };
__constant__ int c_phase_jobs[PH_COUNT][3] = {
    {J_GEOM, J_CLEAR, -1}, {J_DEPOSIT, J_CORNER, -1}, {J_SCANSUM, J_CHMAX, J_CELL}, {J_SCANTOP, J_DCTX, -1},
    {J_SCANAPPLY, J_DCTY, -1}, {J_DCTZ, J_FFTX, -1}, {J_FFTYZ, -1, -1}, {J_FFTXI, -1, -1}, {J_FIELD, -1, -1},
    {J_PUSH, -1, -1}, {J_BOUND, -1, -1}, {J_REDUCE, -1, -1}};
constexpr int h_phase_jobs[PH_COUNT][3] = {
    {J_GEOM, J_CLEAR, -1}, {J_DEPOSIT, J_CORNER, -1}, {J_SCANSUM, J_CHMAX, J_CELL}, {J_SCANTOP, J_DCTX, -1},
    {J_SCANAPPLY, J_DCTY, -1}, {J_DCTZ, J_FFTX, -1}, {J_FFTYZ, -1, -1}, {J_FFTXI, -1, -1}, {J_FIELD, -1, -1},
    {J_PUSH, -1, -1}, {J_BOUND, -1, -1}, {J_REDUCE, -1, -1}};

// What one phase does at kick g (map/kick table entries, push mode, boundary mode)
struct Step {
    int64_t g;
    int kpp;
    int from;       // buffer holding the particles
    int track;      // push: composed map and extrema (else the closing half map)
    int apply;      // boundary: apply the half map of kick g+1 (and track extrema)
    int mom;        // boundary: accumulate moments
    int rec;        // record slot of the reduction
};

template <typename T>
__device__ __forceinline__ int locate(const int* cum, int n_inst, int vb) {
    int lo = 0, hi = n_inst;    // cum[lo] <= vb < cum[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cum[mid] <= vb) lo = mid; else hi = mid;
    }
    return lo;
}

// One function per job, kept out of line so each gets its own register
// allocation instead of one merged allocation for the whole switch.
#define JOB(name) template <typename T> __device__ __noinline__ void name(const Inst<T>& in, int lb, const Step& st)

template <typename T>
__device__ __forceinline__ SortBuf sort_of(const Inst<T>& in, int from) {
    SortBuf sb;
    sb.key = in.key;
    sb.rank = in.rank;
    sb.hist = in.cellcount;
    sb.offs = in.offs;
    sb.ids_in = in.ids[from];
    sb.ids_out = in.ids[1 - from];
    sb.dst = nullptr;
    return sb;
}

JOB(job_geom) { geom_kernel_body<T>(in.mm, in.n, in.n, in.n, in.gamma0, in.geom, in.chmax, kCP, 0, 0, 0, 1); }
JOB(job_clear) {
    const int64_t tot = (int64_t)in.n * in.n * in.n * kCP;
    for (int64_t t = (int64_t)lb * blockDim.x + threadIdx.x; t < tot; t += (int64_t)in.tiles.clear_blocks * blockDim.x)
        in.rho[t] = (T)0;
}
JOB(job_deposit) {
    // warp-sorted deposit, 8 warps of 32 particles per virtual block
    deposit_tile_body<T, kCP, kCP, 8>(in.state[st.from], in.N, in.geom, in.n, in.n, in.n, in.qm, in.rho, in.err,
                                      sort_of(in, st.from), lb);
}
// the near box's corners by a few blocks per instance striding over it (the
// box is a small part of the corner lattice in FP32)
constexpr int kCornerBlocks = 8;
JOB(job_corner) {
    if constexpr (sizeof(T) == 4) green_corner_strided_body(in.geom, in.n, in.n, in.corner, lb, kCornerBlocks);
    else green_corner_kernel_body(in.geom, in.n, in.n, in.n, in.corner, lb, 0, 0, 0);
}
JOB(job_scansum) { scan_sum_kernel_body(in.cellcount, in.n * in.n * in.n, in.bsum, lb, 0, 0, 0); }
JOB(job_chmax) {
    chmax_kernel_body<T>(in.rho, (int64_t)in.n * in.n * in.n, kCP, in.chmax, lb, 0, 0, in.tiles.chmax_blocks);
}
JOB(job_cell) { green_cell_kernel_body<T>(in.geom, in.n, in.n, in.n, in.corner, in.G, lb, 0, 0, 0, 1); }
JOB(job_scantop) {
    scan_top_kernel_body(in.bsum, (in.n * in.n * in.n + kScanChunk - 1) / kScanChunk, 0, 0, 0, 1);
}
JOB(job_scanapply) { scan_apply_kernel_body(in.cellcount, in.n * in.n * in.n, in.bsum, in.offs, lb, 0, 0, 0); }
JOB(job_dctx) { dct_kernel_body<T>(in.G, in.Gtmp, in.dct, in.n + 1, (int64_t)(in.n + 1) * (in.n + 1), lb, 0, 0, 0); }
JOB(job_dcty) { dct_kernel_body<T>(in.Gtmp, in.G, in.dct, in.n + 1, (int64_t)(in.n + 1) * (in.n + 1), lb, 0, 0, 0); }
JOB(job_dctz) { dct_kernel_body<T>(in.G, in.Ghat, in.dct, in.n + 1, (int64_t)(in.n + 1) * (in.n + 1), lb, 0, 0, 0); }
// the slab-path convolution (Ghat stored [kx'][kz'][ky'], see job_cell)
template <typename T, int M>
__device__ __noinline__ void job_fft(int job, const Inst<T>& in, int lb) {
    const FFTDims& d = in.d;
    const int tiles = d.ny / in.yt;
    switch (job) {
        case J_FFTX: fftx_fwd_t_kernel_body<T, M>(in.rho, in.X1, d, in.tw, in.chmax, in.yt, false, lb % tiles, lb / tiles); break;
        case J_FFTYZ: fftyz_kernel_body<T, M, M>(in.X1, in.Ghat, d, in.tw, in.tw, lb % d.Mx, lb / d.Mx); break;
        default: fftx_inv_t_kernel_body<T, M>(in.X1, in.phi, d, in.tw, in.chmax, in.yt, lb % tiles, lb / tiles); break;
    }
}
JOB(job_field) {
    switch (in.tiles.field_per) {        // 256-thread field blocks per virtual block
        case 2: field_multi_body<T, 2>(in.phi, in.geom, in.n, in.n, in.n, kCP, in.E, lb); break;
        case 4: field_multi_body<T, 4>(in.phi, in.geom, in.n, in.n, in.n, kCP, in.E, lb); break;
        case 16: field_multi_body<T, 16>(in.phi, in.geom, in.n, in.n, in.n, kCP, in.E, lb); break;
        default: field_multi_body<T, 8>(in.phi, in.geom, in.n, in.n, in.n, kCP, in.E, lb); break;
    }
}
JOB(job_push_track) {
    const int slot = (int)(st.g % st.kpp);
    push_kernel_body<T, kCP, kCP, true>(in.state[st.from], in.state[1 - st.from], in.N, in.E, in.geom, in.n, in.n,
                                        in.n, in.comp[slot], in.kick[slot], in.mm, in.err, sort_of(in, st.from), lb,
                                        0, 0, 0);
}
JOB(job_push_close) {
    const int slot = (int)(st.g % st.kpp);
    push_kernel_body<T, kCP, kCP, false>(in.state[st.from], in.state[1 - st.from], in.N, in.E, in.geom, in.n, in.n,
                                         in.n, in.half[slot], in.kick[slot], in.mm, in.err, sort_of(in, st.from), lb,
                                         0, 0, 0);
}
JOB(job_bound) {
    const MapCoef<T, kCP>& A = in.half[(st.g + 1) % st.kpp];
    if (st.apply && st.mom)
        boundary_kernel_body<T, kCP, kCP, true, true>(in.state[st.from], in.N, A, in.partial, in.mm, lb, 0, 0,
                                                      in.tiles.bound_blocks);
    else if (st.mom)
        boundary_kernel_body<T, kCP, kCP, true, false>(in.state[st.from], in.N, A, in.partial, in.mm, lb, 0, 0,
                                                       in.tiles.bound_blocks);
    else if (st.apply)
        boundary_kernel_body<T, kCP, kCP, false, true>(in.state[st.from], in.N, A, in.partial, in.mm, lb, 0, 0,
                                                       in.tiles.bound_blocks);
}
JOB(job_reduce) {
    moments_reduce_kernel_body(in.partial, in.tiles.bound_blocks, kCP, in.N, in.records + (int64_t)st.rec * 15 * kCP, lb, 0, 0,
                               0);
}
#undef JOB

template <typename T>
__device__ __forceinline__ void do_job(int job, const Inst<T>& in, int lb, const Step& st) {
    switch (job) {
        case J_GEOM: job_geom<T>(in, lb, st); break;
        case J_CLEAR: job_clear<T>(in, lb, st); break;
        case J_DEPOSIT: job_deposit<T>(in, lb, st); break;
        case J_CORNER: job_corner<T>(in, lb, st); break;
        case J_SCANSUM: job_scansum<T>(in, lb, st); break;
        case J_CHMAX: job_chmax<T>(in, lb, st); break;
        case J_CELL: job_cell<T>(in, lb, st); break;
        case J_SCANTOP: job_scantop<T>(in, lb, st); break;
        case J_DCTX: job_dctx<T>(in, lb, st); break;
        case J_SCANAPPLY: job_scanapply<T>(in, lb, st); break;
        case J_DCTY: job_dcty<T>(in, lb, st); break;
        case J_DCTZ: job_dctz<T>(in, lb, st); break;
        case J_FFTX:
        case J_FFTYZ:
        case J_FFTXI:
            if (in.M == 64) job_fft<T, 64>(job, in, lb);
            else job_fft<T, 128>(job, in, lb);
            break;
        case J_FIELD: job_field<T>(in, lb, st); break;
        case J_PUSH:
            if (st.track) job_push_track<T>(in, lb, st);
            else job_push_close<T>(in, lb, st);
            break;
        case J_BOUND: job_bound<T>(in, lb, st); break;
        default: job_reduce<T>(in, lb, st); break;
    }
}

// the virtual blocks of one phase (all its jobs, all instances), strided by `stride`
template <typename T>
__device__ void run_phase(int ph, const Inst<T>* I, int n_inst, const int* cum, const Step& st, int first,
                          int stride) {
    int total = 0, jobs[3], base[4];
    base[0] = 0;
    int nj = 0;
    for (int q = 0; q < 3; ++q) {
        const int j = c_phase_jobs[ph][q];
        if (j < 0) break;
        jobs[nj] = j;
        total += cum[j * (n_inst + 1) + n_inst];
        base[++nj] = total;
    }
    for (int vb = first; vb < total; vb += stride) {
        int q = 0;
        while (vb >= base[q + 1]) ++q;
        const int* c = cum + jobs[q] * (n_inst + 1);
        const int local = vb - base[q];
        const int inst = locate<T>(c, n_inst, local);
        do_job<T>(jobs[q], I[inst], local - c[inst], st);
        // the next job of this block reuses the same shared memory
        __syncthreads();
    }
}

struct RunSpec {
    int64_t g0;
    int n;
    int kpp;
    int first;
    int from;
};

// the split-step sequence of a run (the same order as the single-instance runtime)
template <typename T, typename Sync>
__device__ void run_sequence(const Inst<T>* I, int n_inst, const int* cum, const RunSpec& rs, int first_vb,
                             int stride, Sync sync) {
    Step st;
    st.kpp = rs.kpp;
    st.from = rs.from;
    st.rec = 0;
    st.track = 0;
    if (rs.n == 0) {
        st.g = rs.g0 - 1;
        st.apply = 0;
        st.mom = 1;
        run_phase<T>(PH_BOUND, I, n_inst, cum, st, first_vb, stride);
        sync();
        run_phase<T>(PH_REDUCE, I, n_inst, cum, st, first_vb, stride);
        return;
    }
    st.g = rs.g0 - 1;      // the boundary applies the half map of kick g + 1 = g0
    st.apply = 1;
    st.mom = rs.first;
    run_phase<T>(PH_BOUND, I, n_inst, cum, st, first_vb, stride);
    sync();
    if (rs.first) {
        run_phase<T>(PH_REDUCE, I, n_inst, cum, st, first_vb, stride);
        sync();
        ++st.rec;
    }
    for (int i = 0; i < rs.n; ++i) {
        st.g = rs.g0 + i;
        const bool last = i == rs.n - 1;
        const bool pend = ((st.g + 1) % rs.kpp) == 0;
        for (int ph = PH_GEOM; ph <= PH_FIELD; ++ph) {
            run_phase<T>(ph, I, n_inst, cum, st, first_vb, stride);
            sync();
        }
        st.track = !(last || pend);
        run_phase<T>(PH_PUSH, I, n_inst, cum, st, first_vb, stride);
        sync();
        st.from = 1 - st.from;
        if (last || pend) {
            st.apply = !last;
            st.mom = 1;
            run_phase<T>(PH_BOUND, I, n_inst, cum, st, first_vb, stride);
            sync();
            run_phase<T>(PH_REDUCE, I, n_inst, cum, st, first_vb, stride);
            sync();
            ++st.rec;
        }
    }
}

template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB)
    batch_persistent_kernel(const Inst<T>* __restrict__ I, int n_inst, const int* __restrict__ cum, RunSpec rs) {
    cg::grid_group grid = cg::this_grid();
    run_sequence<T>(I, n_inst, cum, rs, (int)blockIdx.x, (int)gridDim.x, [&]() { grid.sync(); });
}

// phased mode: one kernel per phase whose jobs are compile-time constants, so
// each kernel holds (and allocates registers for) only its own job bodies
template <typename T, int J>
__device__ __forceinline__ void run_job_blocks(const Inst<T>* I, int n_inst, const int* cum, const Step& st,
                                               int local_vb) {
    const int* c = cum + J * (n_inst + 1);
    const int inst = locate<T>(c, n_inst, local_vb);
    do_job<T>(J, I[inst], local_vb - c[inst], st);
}

// threads per CTA of a phase kernel: the slab FFT phase takes 512 (its bodies
// stride by blockDim), every other phase 256
template <int PH>
__host__ __device__ constexpr int phase_threads() { return PH == PH_FFTYZ ? 512 : 256; }

template <typename T, int PH>
__global__ void __launch_bounds__(phase_threads<PH>(), 2) batch_phase_kernel(const Inst<T>* __restrict__ I, int n_inst,
                                                          const int* __restrict__ cum, Step st) {
    constexpr int J0 = h_phase_jobs[PH][0], J1 = h_phase_jobs[PH][1], J2 = h_phase_jobs[PH][2];
    const int t0 = cum[J0 * (n_inst + 1) + n_inst];
    const int t1 = t0 + (J1 >= 0 ? cum[(J1 >= 0 ? J1 : 0) * (n_inst + 1) + n_inst] : 0);
    const int t2 = t1 + (J2 >= 0 ? cum[(J2 >= 0 ? J2 : 0) * (n_inst + 1) + n_inst] : 0);
    for (int vb = (int)blockIdx.x; vb < t2; vb += (int)gridDim.x) {
        if (vb < t0) run_job_blocks<T, J0>(I, n_inst, cum, st, vb);
        else if constexpr (J1 >= 0) {
            if (vb < t1) run_job_blocks<T, J1>(I, n_inst, cum, st, vb - t0);
            else if constexpr (J2 >= 0) run_job_blocks<T, J2>(I, n_inst, cum, st, vb - t1);
        }
        __syncthreads();
    }
}

template <typename T>
void launch_phase(int ph, int nb, size_t smem, cudaStream_t s, const Inst<T>* I, int n_inst, const int* cum,
                  const Step& st) {
    switch (ph) {
#define ADPIC_PHASE(P) \
    case P: batch_phase_kernel<T, P><<<nb, phase_threads<P>(), smem, s>>>(I, n_inst, cum, st); break;
        ADPIC_PHASE(0) ADPIC_PHASE(1) ADPIC_PHASE(2) ADPIC_PHASE(3) ADPIC_PHASE(4) ADPIC_PHASE(5)
        ADPIC_PHASE(6) ADPIC_PHASE(7) ADPIC_PHASE(8) ADPIC_PHASE(9) ADPIC_PHASE(10) ADPIC_PHASE(11)
#undef ADPIC_PHASE
        default: break;
    }
}

template <typename T, int PH>
void phase_attrs(int mx) {
    cudaFuncSetAttribute(batch_phase_kernel<T, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if constexpr (PH + 1 < PH_COUNT) phase_attrs<T, PH + 1>(mx);
}

// host twin of run_sequence for the phased mode
template <typename T>
void enqueue_phased(const Inst<T>* I, int n_inst, const int* cum, const std::vector<int>& phase_blocks,
                    const RunSpec& rs, const std::vector<size_t>& phase_smem, cudaStream_t s) {
    Step st{};
    st.kpp = rs.kpp;
    st.from = rs.from;
    // each phase launches with the shared memory of its own jobs only
    auto launch = [&](int ph) {
        const int nb = phase_blocks[ph];
        if (nb > 0) launch_phase<T>(ph, nb, phase_smem[ph], s, I, n_inst, cum, st);
    };
    if (rs.n == 0) {
        st.g = rs.g0 - 1;
        st.apply = 0;
        st.mom = 1;
        launch(PH_BOUND);
        launch(PH_REDUCE);
        return;
    }
    st.g = rs.g0 - 1;
    st.apply = 1;
    st.mom = rs.first;
    launch(PH_BOUND);
    if (rs.first) {
        launch(PH_REDUCE);
        ++st.rec;
    }
    for (int i = 0; i < rs.n; ++i) {
        st.g = rs.g0 + i;
        const bool last = i == rs.n - 1;
        const bool pend = ((st.g + 1) % rs.kpp) == 0;
        for (int ph = PH_GEOM; ph <= PH_FIELD; ++ph) launch(ph);
        st.track = !(last || pend);
        launch(PH_PUSH);
        st.from = 1 - st.from;
        if (last || pend) {
            st.apply = !last;
            st.mom = 1;
            launch(PH_BOUND);
            launch(PH_REDUCE);
            ++st.rec;
        }
    }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// ====================================================================== handle

struct ad_pic_batch {
    int n_inst = 0, prec = 0;
    std::vector<ad_pic*> h;
    cudaStream_t stream = nullptr;
    void* inst_dev = nullptr;                 // Inst<T>[n_inst]
    int* cum_dev = nullptr;                   // [J_COUNT][n_inst + 1]
    std::vector<int> phase_blocks;            // virtual blocks per phase
    std::vector<size_t> phase_smem;           // dynamic shared memory per phase (phased mode)
    void* coef_dev = nullptr;                 // per-instance half/comp/kick tables
    size_t coef_bytes = 0;
    double* records = nullptr;                // [n_inst][rec_cap][15][CP]
    int rec_cap = 0;
    int* errs = nullptr;                      // [n_inst]
    void* snapshot = nullptr;                 // autotuner: saved particle buffers
    size_t snapshot_bytes = 0;
    size_t smem = 0;
    int mode = 0;                             // 0 auto, 1/2 persistent (blocks per SM), 3 phased
    int tuned_mode = 0;
    double tune_ms[4] = {0, 0, 0, 0};
    Tiles tiles;                              // tile shapes in use
    bool tiles_fixed = false;                 // set by the caller: the tuner keeps them
    double tiles_ms = 0;                      // kick time with the tuned tiles (0: not tuned)
    bool use_graphs = true;
    std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;
};

namespace {

void batch_free_graphs(ad_pic_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// FFT dimensions of a cubic instance with n^3 nodes
FFTDims h_dims(int n) {
    FFTDims d{};
    d.nx = d.ny = d.nz = n;
    d.Mx = d.My = d.Mz = 2 * n;
    int l = 0;
    while ((1 << l) < 2 * n) ++l;
    d.lx = d.ly = d.lz = l;
    d.C = kCP;
    d.CP = kCP;
    d.npair = kCP / 2;
    d.norm = 1.0 / ((double)(2 * n) * (2 * n) * (2 * n));
    return d;
}

template <typename T>
size_t lane_smem(int n) {
    const size_t dct = sizeof(T) * ((size_t)(n + 1) * (n + 1) + (size_t)kDctLines * (n + 2));
    const size_t dep = 8 * dep_tile_bytes_per_warp<kCP, T>();    // deposit tiles of 8 warps
    const size_t slab = fft_slab_smem<T>(h_dims(n));
    return std::max(std::max(slab, dep), dct);
}

// dynamic shared memory of one job on a cubic n^3 instance
template <typename T>
size_t job_smem(int job, int n) {
    switch (job) {
        case J_DEPOSIT: return 8 * dep_tile_bytes_per_warp<kCP, T>();
        case J_DCTX:
        case J_DCTY:
        case J_DCTZ: return sizeof(T) * ((size_t)(n + 1) * (n + 1) + (size_t)kDctLines * (n + 2));
        case J_FFTX: return fft_slab_smem<T>(h_dims(n), 0);
        case J_FFTYZ: return fft_slab_smem<T>(h_dims(n), 1);
        case J_FFTXI: return fft_slab_smem<T>(h_dims(n), 2);
        default: return 0;
    }
}

template <typename T>
int build_tables(ad_pic_batch* b) {
    const int ni = b->n_inst;
    std::vector<int> blocks((size_t)J_COUNT * ni);
    size_t smem = 0;
    for (int i = 0; i < ni; ++i) {
        ad_pic* h = b->h[i];
        const int n = h->nx;
        const int64_t nodes = (int64_t)n * n * n;
        const int M = 2 * n;
        const int npair = kCP / 2;
        int* bl = blocks.data();
        auto set = [&](int j, int64_t v) { bl[(size_t)j * ni + i] = (int)v; };
        set(J_GEOM, 1);
        set(J_CLEAR, b->tiles.clear_blocks);
        set(J_DEPOSIT, ceil_div(h->N, 256));
        set(J_CORNER, sizeof(T) == 4 ? kCornerBlocks : ceil_div((int64_t)(n + 2) * (n + 2) * (n + 2), 256));
        set(J_SCANSUM, scan_blocks((int)nodes));
        set(J_CHMAX, b->tiles.chmax_blocks);
        set(J_CELL, ceil_div((int64_t)(n + 1) * (n + 1) * (n + 1), 256));
        set(J_SCANTOP, 1);
        set(J_DCTX, ceil_div((int64_t)(n + 1) * (n + 1), kDctLines));
        set(J_SCANAPPLY, scan_blocks((int)nodes));
        set(J_DCTY, ceil_div((int64_t)(n + 1) * (n + 1), kDctLines));
        set(J_DCTZ, ceil_div((int64_t)(n + 1) * (n + 1), kDctLines));
        const int yt = fft_slab_yt<T>(h_dims(n));
        set(J_FFTX, (int64_t)(n / yt) * n);
        set(J_FFTYZ, (int64_t)M * npair);
        set(J_FFTXI, (int64_t)(n / yt) * n);
        set(J_FIELD, ceil_div(nodes * kCP, 256 * b->tiles.field_per));
        set(J_PUSH, ceil_div(h->N, 256));
        set(J_BOUND, b->tiles.bound_blocks);
        set(J_REDUCE, 15 * kCP);
        smem = std::max(smem, lane_smem<T>(n));
    }
    std::vector<int> cum((size_t)J_COUNT * (ni + 1));
    for (int j = 0; j < J_COUNT; ++j) {
        cum[(size_t)j * (ni + 1)] = 0;
        for (int i = 0; i < ni; ++i)
            cum[(size_t)j * (ni + 1) + i + 1] = cum[(size_t)j * (ni + 1) + i] + blocks[(size_t)j * ni + i];
    }
    b->phase_smem.assign(PH_COUNT, 0);
    for (int i = 0; i < ni; ++i)
        for (int ph = 0; ph < PH_COUNT; ++ph)
            for (int q = 0; q < 3; ++q)
                if (h_phase_jobs[ph][q] >= 0)
                    b->phase_smem[ph] = std::max(b->phase_smem[ph], job_smem<T>(h_phase_jobs[ph][q], b->h[i]->nx));
    b->phase_blocks.assign(PH_COUNT, 0);
    for (int ph = 0; ph < PH_COUNT; ++ph)
        for (int q = 0; q < 3; ++q)
            if (h_phase_jobs[ph][q] >= 0) b->phase_blocks[ph] += cum[(size_t)h_phase_jobs[ph][q] * (ni + 1) + ni];
    b->smem = smem;
    if (!b->cum_dev && cudaMalloc(&b->cum_dev, sizeof(int) * cum.size()) != cudaSuccess) {
        cudaGetLastError();
        b->cum_dev = nullptr;
        return AD_PIC_ERR_OOM;
    }
    if (cudaMemcpy(b->cum_dev, cum.data(), sizeof(int) * cum.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    const int mx = 200 * 1024;
    cudaFuncSetAttribute(batch_persistent_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(batch_persistent_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    phase_attrs<T, 0>(mx);
    return AD_PIC_OK;
}

// instance table and coefficient tables on the device (after the handles' tables are built)
template <typename T>
int upload_instances(ad_pic_batch* b, int nrec) {
    const int ni = b->n_inst;
    using MC = MapCoef<T, kCP>;
    using KC = KickCoef<T, kCP>;
    const int kpp = b->h[0]->kpp;
    const size_t per = (2 * sizeof(MC) + sizeof(KC)) * kpp;
    if (per * ni > b->coef_bytes) {
        if (b->coef_dev) cudaFree(b->coef_dev);
        if (cudaMalloc(&b->coef_dev, per * ni) != cudaSuccess) { cudaGetLastError(); b->coef_dev = nullptr; return AD_PIC_ERR_OOM; }
        b->coef_bytes = per * ni;
    }
    if (nrec > b->rec_cap) {
        if (b->records) cudaFree(b->records);
        if (cudaMalloc(&b->records, sizeof(double) * 15 * kCP * (size_t)nrec * ni) != cudaSuccess) {
            cudaGetLastError();
            b->records = nullptr;
            return AD_PIC_ERR_OOM;
        }
        b->rec_cap = nrec;
    }
    std::vector<unsigned char> coef(per * ni);
    std::vector<Inst<T>> I(ni);
    for (int i = 0; i < ni; ++i) {
        ad_pic* h = b->h[i];
        unsigned char* base = coef.data() + per * i;
        std::memcpy(base, h->half.data(), sizeof(MC) * kpp);
        std::memcpy(base + sizeof(MC) * kpp, h->comp.data(), sizeof(MC) * kpp);
        std::memcpy(base + 2 * sizeof(MC) * kpp, h->kcoef.data(), sizeof(KC) * kpp);
        unsigned char* dbase = (unsigned char*)b->coef_dev + per * i;
        Inst<T>& in = I[i];
        in.n = h->nx;
        in.M = 2 * h->nx;
        in.N = h->N;
        in.qm = (T)h->qm;
        in.gamma0 = h->gamma0;
        in.d.nx = in.d.ny = in.d.nz = h->nx;
        in.d.Mx = in.d.My = in.d.Mz = in.M;
        int l = 0;
        while ((1 << l) < in.M) ++l;
        in.d.lx = in.d.ly = in.d.lz = l;
        in.d.C = kCP;
        in.d.CP = kCP;
        in.d.npair = kCP / 2;
        in.d.norm = 1.0 / ((double)in.M * in.M * in.M);
        in.yt = fft_slab_yt<T>(in.d);
        in.state[0] = (T*)h->state;
        in.state[1] = (T*)h->state2;
        in.ids[0] = h->ids[0];
        in.ids[1] = h->ids[1];
        in.key = h->key;
        in.rank = h->rank;
        in.cellcount = h->cellcount;
        in.offs = h->offs;
        in.bsum = h->bsum;
        in.rho = (T*)h->rho;
        in.phi = (T*)h->phi;
        in.E = (T*)h->E;
        in.X1 = (V2<T>*)h->X1;
        in.X2 = (V2<T>*)h->X2;
        in.G = (T*)h->G;
        in.Gtmp = (T*)h->Gtmp;
        in.Ghat = (T*)h->Ghat;
        in.corner = h->corner;
        in.dct = (const T*)h->dct[0];
        in.tw = (const V2<T>*)h->tw[0];
        in.geom = h->geom;
        in.mm = (Ord<T>*)h->mm;
        in.chmax = (Ord<T>*)h->chmax;
        in.err = b->errs + i;
        in.partial = h->partial;
        in.records = b->records + (size_t)i * b->rec_cap * 15 * kCP;
        in.half = (const MC*)dbase;
        in.comp = (const MC*)(dbase + sizeof(MC) * kpp);
        in.kick = (const KC*)(dbase + 2 * sizeof(MC) * kpp);
        in.tiles = b->tiles;
    }
    if (!b->inst_dev && cudaMalloc(&b->inst_dev, sizeof(Inst<T>) * ni) != cudaSuccess) {
        cudaGetLastError();
        b->inst_dev = nullptr;
        return AD_PIC_ERR_OOM;
    }
    if (cudaMemcpyAsync(b->coef_dev, coef.data(), coef.size(), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->inst_dev, I.data(), sizeof(Inst<T>) * ni, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return AD_PIC_ERR_CUDA;
    return AD_PIC_OK;
}

template <typename T>
int launch_mode(ad_pic_batch* b, int mode, const RunSpec& rs) {
    const Inst<T>* I = (const Inst<T>*)b->inst_dev;
    if (mode == 3) {
        enqueue_phased<T>(I, b->n_inst, b->cum_dev, b->phase_blocks, rs, b->phase_smem, b->stream);
        return cudaGetLastError() == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* fn = mode == 2 ? (void*)batch_persistent_kernel<T, 2> : (void*)batch_persistent_kernel<T, 1>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, b->smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return AD_PIC_ERR_UNSUPPORTED;
    }
    per_sm = std::min(per_sm, mode == 2 ? 2 : 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * per_sm));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int ni = b->n_inst;
    const int* cum = b->cum_dev;
    cudaError_t e = mode == 2 ? cudaLaunchKernelEx(&cfg, batch_persistent_kernel<T, 2>, I, ni, cum, rs)
                              : cudaLaunchKernelEx(&cfg, batch_persistent_kernel<T, 1>, I, ni, cum, rs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AD_PIC_ERR_CUDA;
    }
    return AD_PIC_OK;
}

template <typename T>
int enqueue(ad_pic_batch* b, int mode, const RunSpec& rs) {
    if (cudaMemsetAsync(b->errs, 0, sizeof(int) * b->n_inst, b->stream) != cudaSuccess) return AD_PIC_ERR_CUDA;
    return launch_mode<T>(b, mode, rs);
}

// time one kick of the real batch in each mode on a snapshot of the particles and
// keep the fastest; then, in that mode, a coordinate search over the tile shapes
// (each shape in turn over its choices, the others held), keeping the fastest
template <typename T>
int autotune_measure(ad_pic_batch* b, const RunSpec& base, int nrec) {
    size_t need = 0;
    for (ad_pic* h : b->h) need += sizeof(T) * 6 * h->N * kCP;
    if (need > b->snapshot_bytes) {
        if (b->snapshot) cudaFree(b->snapshot);
        if (cudaMalloc(&b->snapshot, need) != cudaSuccess) {
            cudaGetLastError();
            b->snapshot = nullptr;
            b->tuned_mode = 3;
            return AD_PIC_OK;
        }
        b->snapshot_bytes = need;
    }
    auto copy = [&](bool save) {
        size_t off = 0;
        for (ad_pic* h : b->h) {
            const size_t bytes = sizeof(T) * 6 * h->N * kCP;
            void* cur = h->cur ? h->state2 : h->state;
            char* snap = (char*)b->snapshot + off;
            cudaMemcpyAsync(save ? snap : cur, save ? cur : snap, bytes, cudaMemcpyDeviceToDevice, b->stream);
            off += bytes;
        }
    };
    RunSpec rs = base;
    rs.n = 1;
    rs.first = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    copy(true);
    auto time_kick = [&](int mode, bool& ok) -> float {
        float ms = 0.f;
        ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {       // the first repetition warms up
            cudaEventRecord(e0, b->stream);
            ok = enqueue<T>(b, mode, rs) == AD_PIC_OK;
            cudaEventRecord(e1, b->stream);
            ok = ok && cudaStreamSynchronize(b->stream) == cudaSuccess;
            cudaEventElapsedTime(&ms, e0, e1);
            copy(false);
        }
        cudaGetLastError();
        return ms;
    };
    float best = 1e30f;
    int best_mode = 3;
    for (int mode = 1; mode <= 3; ++mode) {
        bool ok = true;
        const float ms = time_kick(mode, ok);
        b->tune_ms[mode] = ok ? ms : -1.0;
        if (ok && ms < best) {
            best = ms;
            best_mode = mode;
        }
    }
    b->tuned_mode = best_mode;
    int rc = AD_PIC_OK;
    if (!b->tiles_fixed) {
        int* knob[4] = {&b->tiles.bound_blocks, &b->tiles.chmax_blocks, &b->tiles.clear_blocks, &b->tiles.field_per};
        for (int j = 0; j < 4 && !rc; ++j) {
            const int keep = *knob[j];
            int best_v = keep;
            for (int c = 0; c < 4 && !rc; ++c) {
                const int v = kTileChoices[j][c];
                if (v == keep) continue;
                *knob[j] = v;
                rc = build_tables<T>(b);
                if (!rc) rc = upload_instances<T>(b, nrec);
                if (rc) break;
                bool ok = true;
                const float ms = time_kick(best_mode, ok);
                if (ok && ms < best) {
                    best = ms;
                    best_v = v;
                }
            }
            *knob[j] = best_v;
        }
        if (!rc) rc = build_tables<T>(b);
        if (!rc) rc = upload_instances<T>(b, nrec);
        b->tiles_ms = best;
    }
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Tuned modes of earlier batches with the same composition (grid size and
// particle-count octave of every instance) on the same device: a batch like
// one already timed reuses its choice instead of timing the modes again.
struct TuneEntry {
    int mode;
    double ms[4];
    Tiles tiles;
    double tiles_ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;

std::string tune_key(const ad_pic_batch* b) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::map<std::pair<int, int>, int> counts;
    for (const ad_pic* h : b->h) {
        int oct = 0;
        while (((int64_t)1 << (oct + 1)) <= h->N) ++oct;
        counts[{h->nx, oct}]++;
    }
    std::string k = std::to_string(dev) + "|" + std::to_string(b->h[0]->prec) + "|";
    for (const auto& kv : counts)
        k += std::to_string(kv.first.first) + "/" + std::to_string(kv.first.second) + "x" + std::to_string(kv.second) + ";";
    return k;
}

template <typename T>
int autotune(ad_pic_batch* b, const RunSpec& base, int nrec) {
    const std::string key = tune_key(b) + (b->tiles_fixed ? "|fixed" : "");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->tuned_mode = it->second.mode;
            for (int m = 0; m < 4; ++m) b->tune_ms[m] = it->second.ms[m];
            if (!b->tiles_fixed) {
                b->tiles = it->second.tiles;
                b->tiles_ms = it->second.tiles_ms;
                int rc = build_tables<T>(b);
                if (!rc) rc = upload_instances<T>(b, nrec);
                return rc;
            }
            return AD_PIC_OK;
        }
    }
    const int st = autotune_measure<T>(b, base, nrec);
    if (st) return st;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    TuneEntry e;
    e.mode = b->tuned_mode;
    for (int m = 0; m < 4; ++m) e.ms[m] = b->tune_ms[m];
    e.tiles = b->tiles;
    e.tiles_ms = b->tiles_ms;
    g_tune_cache[key] = e;
    return st;
}

template <typename T>
int batch_run(ad_pic_batch* b, int n) {
    const int ni = b->n_inst;
    int nrec = 0;
    for (int i = 0; i < ni; ++i) {
        ad_pic* h = b->h[i];
        if (!h->beam_set || !h->lattice_set || !h->particles_set) return AD_PIC_ERR_STATE;
        int r = 0;
        int st = adpic_prepare_run(h, n, &r);
        if (st) return st;
        if (i == 0) nrec = r;
        if (r != nrec || h->kpp != b->h[0]->kpp || h->kick != b->h[0]->kick || h->cur != b->h[0]->cur ||
            h->first_record != b->h[0]->first_record)
            return AD_PIC_ERR_STATE;
    }
    int st = upload_instances<T>(b, std::max(nrec, 1));
    if (st) return st;
    ad_pic* h0 = b->h[0];
    RunSpec rs;
    rs.g0 = h0->kick;
    rs.n = n;
    rs.kpp = h0->kpp;
    rs.first = h0->first_record ? 1 : 0;
    rs.from = h0->cur;
    int mode = b->mode;
    if (mode == 0) {
        if (!b->tuned_mode && n > 0) {
            st = autotune<T>(b, rs, std::max(nrec, 1));
            if (st) return st;
        }
        mode = b->tuned_mode ? b->tuned_mode : 3;
    }
    if (b->use_graphs) {
        auto key = std::make_tuple((int)(rs.g0 % rs.kpp), n, rs.first, rs.from, mode);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AD_PIC_ERR_CUDA;
            int est = enqueue<T>(b, mode, rs);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
            if (est || ce != cudaSuccess) {
                cudaGetLastError();
                b->use_graphs = false;       // fall back to direct launches
            } else {
                cudaGraphExec_t ex;
                if (cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphDestroy(graph);
                    b->use_graphs = false;
                } else {
                    cudaGraphDestroy(graph);
                    it = b->graphs.emplace(key, ex).first;
                }
            }
        }
        if (b->use_graphs) {
            if (cudaGraphLaunch(it->second, b->stream) != cudaSuccess) return AD_PIC_ERR_CUDA;
        } else {
            st = enqueue<T>(b, mode, rs);
            if (st) return st;
        }
    } else {
        st = enqueue<T>(b, mode, rs);
        if (st) return st;
    }
    std::vector<double> rec((size_t)ni * b->rec_cap * 15 * kCP);
    std::vector<int> errs(ni);
    if (cudaMemcpyAsync(rec.data(), b->records, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(errs.data(), b->errs, sizeof(int) * ni, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return AD_PIC_ERR_CUDA;
    }
    int worst = 0;
    for (int i = 0; i < ni; ++i) {
        adpic_finish_run(b->h[i], rec.data() + (size_t)i * b->rec_cap * 15 * kCP, nrec, n);
        worst |= errs[i];
    }
    if (worst & kErrNonfinite) return AD_PIC_ERR_NONFINITE;
    if (worst & kErrOutOfGrid) return AD_PIC_ERR_OUT_OF_GRID;
    return AD_PIC_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int ad_pic_batch_create(int n_inst, const ad_pic_grid* grids, const int64_t* n_particles, int n_deriv, int precision,
                        ad_pic_batch** out) {
    if (!out) return AD_PIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_inst < 1 || n_inst > 65536 || !grids || !n_particles || n_deriv != 7) return AD_PIC_ERR_INVALID_ARG;
    if (precision != AD_PIC_FP32_MIXED) return AD_PIC_ERR_UNSUPPORTED;
    for (int i = 0; i < n_inst; ++i) {
        const ad_pic_grid& g = grids[i];
        if (g.nx != g.ny || g.nx != g.nz || (g.nx != 32 && g.nx != 64)) return AD_PIC_ERR_INVALID_ARG;
        if (n_particles[i] < 1 || n_particles[i] > ((int64_t)1 << 31) - 1) return AD_PIC_ERR_INVALID_ARG;
    }
    ad_pic_batch* b = new (std::nothrow) ad_pic_batch();
    if (!b) return AD_PIC_ERR_OOM;
    b->n_inst = n_inst;
    b->prec = precision;
    b->h.assign(n_inst, nullptr);
    int st = AD_PIC_OK;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) st = AD_PIC_ERR_CUDA;
    for (int i = 0; i < n_inst && !st; ++i) {
        st = ad_pic_create(&grids[i], n_particles[i], n_deriv, precision, &b->h[i]);
        if (!st) ad_pic_set_stream(b->h[i], b->stream);
    }
    if (!st && cudaMalloc(&b->errs, sizeof(int) * n_inst) != cudaSuccess) {
        cudaGetLastError();
        st = AD_PIC_ERR_OOM;
    }
    if (!st) st = build_tables<float>(b);
    if (st) {
        ad_pic_batch_destroy(b);
        return st;
    }
    *out = b;
    return AD_PIC_OK;
}

int ad_pic_batch_set_beam(ad_pic_batch* b, int inst, const ad_pic_beam* beam, const double* normals) {
    if (!b || inst < 0 || inst >= b->n_inst || !beam) return AD_PIC_ERR_INVALID_ARG;
    if (beam->charge_deriv_slot != -1) return AD_PIC_ERR_UNSUPPORTED;   // the batched deposit has no charge channel
    if (beam->energy_deriv_slot != -1) return AD_PIC_ERR_UNSUPPORTED;   // nor the energy term of the convolution
    batch_free_graphs(b);
    return ad_pic_set_beam(b->h[inst], beam, normals);
}

int ad_pic_batch_set_particles(ad_pic_batch* b, int inst, const double* state) {
    if (!b || inst < 0 || inst >= b->n_inst) return AD_PIC_ERR_INVALID_ARG;
    return ad_pic_set_particles(b->h[inst], state);
}

int ad_pic_batch_set_lattice(ad_pic_batch* b, int inst, const ad_pic_lattice* lattice) {
    if (!b || inst < 0 || inst >= b->n_inst) return AD_PIC_ERR_INVALID_ARG;
    batch_free_graphs(b);
    return ad_pic_set_lattice(b->h[inst], lattice);
}

int ad_pic_batch_run(ad_pic_batch* b, int n_steps) {
    if (!b || n_steps < 0) return AD_PIC_ERR_INVALID_ARG;
    return batch_run<float>(b, n_steps);
}

int ad_pic_batch_moments(const ad_pic_batch* b, int inst, double* values, double* derivs) {
    if (!b || inst < 0 || inst >= b->n_inst) return AD_PIC_ERR_INVALID_ARG;
    return ad_pic_moments(b->h[inst], values, derivs);
}

int ad_pic_batch_history(const ad_pic_batch* b, int inst, double* hist, int max_records, int* n_records) {
    if (!b || inst < 0 || inst >= b->n_inst) return AD_PIC_ERR_INVALID_ARG;
    return ad_pic_history(b->h[inst], hist, max_records, n_records);
}

int ad_pic_batch_get_particles(const ad_pic_batch* b, int inst, double* state) {
    if (!b || inst < 0 || inst >= b->n_inst) return AD_PIC_ERR_INVALID_ARG;
    return ad_pic_get_particles(b->h[inst], state);
}

int ad_pic_batch_set_mode(ad_pic_batch* b, int mode) {
    if (!b || mode < 0 || mode > 3) return AD_PIC_ERR_INVALID_ARG;
    b->mode = mode;
    return AD_PIC_OK;
}

int ad_pic_batch_tuning(const ad_pic_batch* b, int* mode, double* ms) {
    if (!b) return AD_PIC_ERR_INVALID_ARG;
    if (mode) *mode = b->mode ? b->mode : b->tuned_mode;
    if (ms)
        for (int m = 0; m < 3; ++m) ms[m] = b->tune_ms[m + 1];
    return AD_PIC_OK;
}

int ad_pic_batch_set_tiles(ad_pic_batch* b, const int* tiles) {
    if (!b) return AD_PIC_ERR_INVALID_ARG;
    Tiles t;
    if (tiles) {
        if (tiles[0] < 1 || tiles[0] > 1024 || tiles[1] < 1 || tiles[1] > 64 || tiles[2] < 1 || tiles[2] > 64 ||
            (tiles[3] != 2 && tiles[3] != 4 && tiles[3] != 8 && tiles[3] != 16))
            return AD_PIC_ERR_INVALID_ARG;
        t.bound_blocks = tiles[0];
        t.chmax_blocks = tiles[1];
        t.clear_blocks = tiles[2];
        t.field_per = tiles[3];
    }
    b->tiles = t;
    b->tiles_fixed = tiles != nullptr;
    b->tuned_mode = 0;                        // tune again (the mode) on the next run
    b->tiles_ms = 0;
    batch_free_graphs(b);
    const int st = b->prec == AD_PIC_FP32_MIXED ? build_tables<float>(b) : AD_PIC_ERR_UNSUPPORTED;
    return st;
}

int ad_pic_batch_tiles(const ad_pic_batch* b, int* tiles, double* ms) {
    if (!b || !tiles) return AD_PIC_ERR_INVALID_ARG;
    tiles[0] = b->tiles.bound_blocks;
    tiles[1] = b->tiles.chmax_blocks;
    tiles[2] = b->tiles.clear_blocks;
    tiles[3] = b->tiles.field_per;
    if (ms) *ms = b->tiles_ms;
    return AD_PIC_OK;
}

int ad_pic_batch_set_stream(ad_pic_batch* b, void* stream) {
    if (!b) return AD_PIC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return AD_PIC_ERR_CUDA;
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : b->stream;
    for (ad_pic* h : b->h) ad_pic_set_stream(h, s);
    b->stream = s;
    batch_free_graphs(b);
    return AD_PIC_OK;
}

void ad_pic_batch_destroy(ad_pic_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_graphs(b);
    for (ad_pic* h : b->h)
        if (h) ad_pic_destroy(h);
    cudaFree(b->inst_dev);
    cudaFree(b->cum_dev);
    cudaFree(b->coef_dev);
    cudaFree(b->records);
    cudaFree(b->errs);
    cudaFree(b->snapshot);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
