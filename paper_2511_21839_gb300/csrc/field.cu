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
    template void setup_green<T>();
ADPIC_FIELD_INST(float)
ADPIC_FIELD_INST(double)


}  // namespace adpic
