// Instantiations of the joint bilateral filter kernel for the up stage
// (radii 1-3).
#include "jbf_core.cuh"

namespace dz {

namespace {
template <int R>
struct Kp { static constexpr int value = 4; };

template <int R>
cudaError_t go(const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s) {
    jbf_kernel<JBF_UP, R, Kp<R>::value><<<grid, 256, 0, s>>>(b, a);
    return cudaGetLastError();
}

template <int R>
int occ() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, jbf_kernel<JBF_UP, R, Kp<R>::value>, 256, 0);
    return n > 0 ? n : 1;
}
}  // namespace

cudaError_t launch_jbf_up(int radius, const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s) {
    switch (radius) {
    case 1: return go<1>(b, a, grid, s);
    case 2: return go<2>(b, a, grid, s);
    case 3: return go<3>(b, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_jbf_up(int radius) {
    switch (radius) {
    case 1: return occ<1>();
    case 2: return occ<2>();
    case 3: return occ<3>();
    default: return 1;
    }
}

int kp_jbf_up(int radius) {
    switch (radius) {
    case 1: return Kp<1>::value;
    case 2: return Kp<2>::value;
    case 3: return Kp<3>::value;
    default: return 0;
    }
}

}  // namespace dz
