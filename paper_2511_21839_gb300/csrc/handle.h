// Private: the ad_pic handle, shared by the single-instance runtime (api.cu)
// and the batched runtime (batch.cu). Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <map>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "ad_pic.h"
#include "common.cuh"

constexpr int kClasses = 8;    // kernel classes of the event timing

struct ad_pic {
    using GeomDev = adpic::GeomDev;
    int prec = 0, P = 7, C = 8, CP = 8;
    int nx = 0, ny = 0, nz = 0;
    int64_t N = 0;
    bool beam_set = false, particles_set = false, lattice_set = false, coef_dirty = true;
    double gamma0 = 0, beta0 = 0, p0 = 0, brho = 0, kperp = 0, kz = 0, qm = 0, q = 0;
    int qslot = -1;               // derivative slot of the bunch charge (-1: constant)
    int eslot = -1;               // derivative slot of the kinetic energy (-1: constant)
    double mass_eV = 0;           // rest energy: d gamma0 / dE = 1 / mass_eV
    // the energy's term of the convolution, allocated with the first energy slot:
    // dF/dhzr at the Green's corners, the spectrum of dG/dE, and the two-channel
    // records [node][2] of rho_0 and of (dG/dE) * rho_0
    double* corner_e = nullptr;
    void* Ghat_e = nullptr;
    void* rho_e = nullptr;
    void* phi_e = nullptr;
    ad_pic_lattice lat{};
    // a general beamline in place of the FODO period (empty: the FODO lattice)
    std::vector<ad_pic_element> line;
    std::vector<int> line_kicks;
    int kpp = 0;
    int64_t kick = 0;
    bool first_record = true;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    // the Green's function depends on the grid geometry only: it runs on a side
    // stream concurrently with deposit and channel maxima (fork after the
    // kernel whose last block derived the geometry, join before the
    // convolution). The cell-offset scan is
    // needed by the push only: it follows on the side stream after the deposit
    // (ev_dep) and joins before the push (ev_scan). Captured graphs keep the branches.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_dep = nullptr, ev_scan = nullptr;
    // device memory
    void* state = nullptr;
    void* state2 = nullptr;      // the other buffer of the cell-sorting push
    int cur = 0;                 // which buffer holds the particles (0: state, 1: state2)
    int* ids[2] = {nullptr, nullptr};   // caller's particle index of each slot
    int* key = nullptr;          // cell of each particle at the last deposit
    int* rank = nullptr;         // rank among that cell's particles
    int* cellcount = nullptr;    // particles per cell (zero between kicks)
    int* offs = nullptr;         // exclusive cell offsets
    int* dst = nullptr;          // destination slot of every particle in the push (N + 4 entries)
    int* bsum = nullptr;         // scan chunk totals
    void* rho = nullptr;         // zero between kicks: the convolution's x pass clears it
    unsigned* gcount = nullptr;  // finished blocks of a kernel with the fused geometry step
    void* phi = nullptr;
    void* E = nullptr;
    void* X1 = nullptr;
    void* X2 = nullptr;
    void* G = nullptr;
    void* Gtmp = nullptr;
    void* Ghat = nullptr;
    double* corner = nullptr;
    void* dct[3] = {nullptr, nullptr, nullptr};
    void* tw[3] = {nullptr, nullptr, nullptr};
    GeomDev* geom = nullptr;
    void* mm = nullptr;
    void* chmax = nullptr;
    int* err = nullptr;
    double* partial = nullptr;
    double* records = nullptr;
    int records_cap = 0;
    double* staging = nullptr;      // FP64 [6][N][C] staging buffer of set/get_particles
    // asynchronous FP32 upload (prefetch / commit): its device buffer [6][N][C],
    // the copy stream, the copy's completion and the commit's last read of the buffer
    float* prefetch = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_copied = nullptr, ev_consumed = nullptr;
    bool prefetched = false;
    int64_t launches = 0;           // kernels launched by ad_pic_run so far
    int wait_polls = -1;            // poll limit of the push's tile waits (< 0: the default)
    std::vector<void*> allocs;
    // per-kick coefficients of the handle's precision (raw MapCoef / KickCoef)
    std::vector<unsigned char> half, comp, kcoef;
    std::vector<double> hist;   // records [3][5][C]
    // graphs
    bool use_graphs = true;
    std::map<std::tuple<int, int, int, unsigned, int>, cudaGraphExec_t> graphs;
    // timing
    unsigned tmask = 0;
    std::vector<cudaEvent_t> events;
    std::vector<int> ev_class;
    int ev_used = 0;
    double tms[kClasses] = {0};
    int64_t tcount[kClasses] = {0};
};


// Internal hooks used by the batched runtime (implemented in api.cu).
// Prepare a handle for a run of n_steps kicks driven from outside: per-kick
// coefficient tables built, record buffer large enough; returns a status.
int adpic_prepare_run(ad_pic* h, int n_steps, int* n_records);
// After an outside run: append its moment records [nrec][15][CP] (host
// copy) to the history and advance the kick counter and the buffer parity.
void adpic_finish_run(ad_pic* h, const double* rec, int nrec, int n_steps);
