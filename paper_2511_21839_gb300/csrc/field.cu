// Grid-side kernels: per-kick geometry, the integrated Green's function and
// its real even spectrum, the zero-padded (Hockney) FFT convolution of all
// dual channels, and the central finite-difference field.
#include <algorithm>

#include "field_dev.cuh"

namespace adpic {

template <typename T>
void launch_chmax(const T* rho, int64_t nodes, int CP, Ord<T>* chmax, cudaStream_t s) {
    // rho is cudaMalloc'ed (256-byte aligned) with CP in {8, 16}
    if (CP == 8)
        chmax_vec_kernel<T, 8><<<152 * 2, 256, 0, s>>>(rho, nodes, chmax);
    else if (CP == 16)
        chmax_vec_kernel<T, 16><<<152 * 2, 256, 0, s>>>(rho, nodes, chmax);
    else
        chmax_kernel<T><<<152 * 2, 256, 0, s>>>(rho, nodes, CP, chmax);
}

template <typename T>
void launch_green(const GeomDev* geom, int nx, int ny, int nz, bool exact, double* corner, T* G, T* Gtmp, T* Ghat,
                  const T* dct_x, const T* dct_y, const T* dct_z, int order, cudaStream_t s) {
    (void)exact;
    // FP32: the near box is a small part of the corner lattice, so a fixed grid
    // of 608 blocks strides over it; FP64 (box = whole lattice): one thread per corner
    const int64_t nc = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
    if (sizeof(T) == 4)
        green_corner_strided_kernel<<<(unsigned)std::min<int64_t>((nc + 63) / 64, 152 * 4), 64, 0, s>>>(geom, nx, ny,
                                                                                                      nz, corner);
    else
        green_corner_kernel<<<(unsigned)((nc + 63) / 64), 64, 0, s>>>(geom, nx, ny, nz, corner);
    // each pass transforms the contiguous axis and makes it the outermost one;
    // the first pass computes its lines as the cell averages of G itself (G is
    // never stored). 16 warps per block and ACC = ceil(L / 16) accumulators:
    // the warps cover all L = n + 1 outputs in one sweep
    auto pass = [&](const T* in, T* out, const T* D, int L, int64_t BA, bool cell) {
        const size_t sm = sizeof(T) * ((size_t)L * L + (size_t)kDctLines * L);
        const unsigned grid = (unsigned)((BA + kDctLines - 1) / kDctLines);
#define ADPIC_DCT_PASS(ACC)                                                                                  \
    if (cell)                                                                                                \
        cell_dct_kernel<T, ACC><<<grid, 512, sm, s>>>(out, D, L, BA, geom, nx, ny, nz, corner, order);       \
    else                                                                                                     \
        dct_kernel<T, ACC><<<grid, 512, sm, s>>>(in, out, D, L, BA);
        if (L <= 17) {
            ADPIC_DCT_PASS(2)
        } else if (L <= 33) {
            ADPIC_DCT_PASS(3)
        } else if (L <= 65) {
            ADPIC_DCT_PASS(5)
        } else {
            ADPIC_DCT_PASS(9)
        }
#undef ADPIC_DCT_PASS
    };
    if (order == 0) {
        // G [z][y][x] -> pass x -> [x'][z][y] -> pass y -> [y'][x'][z] -> pass z -> [z'][y'][x']
        pass(nullptr, Gtmp, dct_x, nx + 1, (int64_t)(nz + 1) * (ny + 1), true);
        pass(Gtmp, G, dct_y, ny + 1, (int64_t)(nx + 1) * (nz + 1), false);
        pass(G, Ghat, dct_z, nz + 1, (int64_t)(ny + 1) * (nx + 1), false);
    } else {
        // G [x][z][y] -> pass y -> [y'][x][z] -> pass z -> [z'][y'][x] -> pass x -> [x'][z'][y']
        pass(nullptr, Gtmp, dct_y, ny + 1, (int64_t)(nx + 1) * (nz + 1), true);
        pass(Gtmp, G, dct_z, nz + 1, (int64_t)(ny + 1) * (nx + 1), false);
        pass(G, Ghat, dct_x, nx + 1, (int64_t)(nz + 1) * (ny + 1), false);
    }
}

// dG/dE (the kinetic energy as a dual input) through the same three DCT-I
// passes: dF/dhzr at the corners of the near box, then the cell values of
// dG/dE inside the first pass. F (the corner values of the same geometry)
// must have been computed by launch_green before, on the same stream; G and
// Gtmp are scratch, as there.
template <typename T>
void launch_green_energy(const GeomDev* geom, int nx, int ny, int nz, const double* corner, double* corner_e, T* G,
                         T* Gtmp, T* Ghat_e, const T* dct_x, const T* dct_y, const T* dct_z, int order,
                         double inv_mass_eV, cudaStream_t s) {
    const int64_t nc = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
    green_corner_dz_kernel<<<(unsigned)std::min<int64_t>((nc + 63) / 64, 152 * 4), 64, 0, s>>>(geom, nx, ny, nz,
                                                                                               corner_e);
    auto pass = [&](const T* in, T* out, const T* D, int L, int64_t BA, bool cell) {
        const size_t sm = sizeof(T) * ((size_t)L * L + (size_t)kDctLines * L);
        const unsigned grid = (unsigned)((BA + kDctLines - 1) / kDctLines);
#define ADPIC_DCTE_PASS(ACC)                                                                                 \
    if (cell)                                                                                                \
        cell_dct_energy_kernel<T, ACC><<<grid, 512, sm, s>>>(out, D, L, BA, geom, nx, ny, nz, corner, corner_e, \
                                                             inv_mass_eV, order);                            \
    else                                                                                                     \
        dct_kernel<T, ACC><<<grid, 512, sm, s>>>(in, out, D, L, BA);
        if (L <= 17) {
            ADPIC_DCTE_PASS(2)
        } else if (L <= 33) {
            ADPIC_DCTE_PASS(3)
        } else if (L <= 65) {
            ADPIC_DCTE_PASS(5)
        } else {
            ADPIC_DCTE_PASS(9)
        }
#undef ADPIC_DCTE_PASS
    };
    if (order == 0) {
        pass(nullptr, Gtmp, dct_x, nx + 1, (int64_t)(nz + 1) * (ny + 1), true);
        pass(Gtmp, G, dct_y, ny + 1, (int64_t)(nx + 1) * (nz + 1), false);
        pass(G, Ghat_e, dct_z, nz + 1, (int64_t)(ny + 1) * (nx + 1), false);
    } else {
        pass(nullptr, Gtmp, dct_y, ny + 1, (int64_t)(nx + 1) * (nz + 1), true);
        pass(Gtmp, G, dct_z, nz + 1, (int64_t)(ny + 1) * (nx + 1), false);
        pass(G, Ghat_e, dct_x, nx + 1, (int64_t)(nz + 1) * (ny + 1), false);
    }
}

// channel 0 of rho into the two-channel records of the energy term's
// convolution (the second channel zero: the pair's imaginary half)
template <typename T>
static __global__ void energy_copy_kernel(const T* __restrict__ rho, int CP, int64_t nodes, T* __restrict__ rho_e) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nodes) return;
    rho_e[2 * t] = rho[t * CP];
    rho_e[2 * t + 1] = (T)0;
}
// phi channel ce += (dG/dE) * rho_0 (channel 0 of the energy term's records)
template <typename T>
static __global__ void energy_add_kernel(const T* __restrict__ phi_e, int64_t nodes, T* __restrict__ phi, int CP,
                                         int ce) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nodes) return;
    phi[t * CP + ce] += phi_e[2 * t];
}
// E_z of the energy channel: the field kernel divides by the value of the
// rest-frame spacing 2 gamma0 hz; its energy derivative (Eq. 3 on the
// quotient) adds -E_z,0 (d gamma0/dE) / gamma0 = -r E_z,0
template <typename T>
static __global__ void energy_field_kernel(T* __restrict__ E, int64_t nodes, int CP, int ce, T r) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nodes) return;
    T* ez = E + (t * 3 + 2) * CP;
    ez[ce] -= r * ez[0];
}
template <typename T>
void launch_energy_field(T* E, int64_t nodes, int CP, int ce, double r, cudaStream_t s) {
    energy_field_kernel<T><<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(E, nodes, CP, ce, (T)r);
}
template <typename T>
void launch_energy_copy(const T* rho, int CP, int64_t nodes, T* rho_e, cudaStream_t s) {
    energy_copy_kernel<T><<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(rho, CP, nodes, rho_e);
}
template <typename T>
void launch_energy_add(const T* phi_e, int64_t nodes, T* phi, int CP, int ce, cudaStream_t s) {
    energy_add_kernel<T><<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(phi_e, nodes, phi, CP, ce);
}

template <typename T>
void setup_green() {
    cudaFuncSetAttribute(dct_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(dct_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(dct_kernel<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(dct_kernel<T, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_kernel<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_kernel<T, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_energy_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_energy_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_energy_kernel<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(cell_dct_energy_kernel<T, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T>
void launch_field(const T* phi, const GeomDev* geom, int nx, int ny, int nz, int CP, T* E, cudaStream_t s) {
    // one thread per 32-byte piece of a node's channels (CP in {8, 16})
    const int64_t pieces = (int64_t)nx * ny * nz * CP * (int64_t)sizeof(T) / 32;
    const unsigned grid = (unsigned)((pieces + 255) / 256);
    if (CP == 8)
        field_vec_kernel<T, 8><<<grid, 256, 0, s>>>(phi, geom, nx, ny, nz, E);
    else if (CP == 16)
        field_vec_kernel<T, 16><<<grid, 256, 0, s>>>(phi, geom, nx, ny, nz, E);
    else {
        const int64_t tot = (int64_t)nx * ny * nz * CP;
        field_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(phi, geom, nx, ny, nz, CP, E);
    }
}

#define ADPIC_FIELD_INST(T)                                                                                       \
    template void launch_chmax<T>(const T*, int64_t, int, Ord<T>*, cudaStream_t);                                 \
    template void launch_green<T>(const GeomDev*, int, int, int, bool, double*, T*, T*, T*, const T*, const T*,    \
                                  const T*, int, cudaStream_t);                                                   \
    template void launch_field<T>(const T*, const GeomDev*, int, int, int, int, T*, cudaStream_t);             \
    template void launch_green_energy<T>(const GeomDev*, int, int, int, const double*, double*, T*, T*, T*,      \
                                         const T*, const T*, const T*, int, double, cudaStream_t);                \
    template void launch_energy_copy<T>(const T*, int, int64_t, T*, cudaStream_t);                             \
    template void launch_energy_add<T>(const T*, int64_t, T*, int, int, cudaStream_t);                          \
    template void launch_energy_field<T>(T*, int64_t, int, int, double, cudaStream_t);                          \
    template void setup_green<T>();
ADPIC_FIELD_INST(float)
ADPIC_FIELD_INST(double)


}  // namespace adpic
