// zncc_row.cu -- instantiates k_zncc_row (and the progressive-scan k_zncc_scan and tensor-core k_zncc_mma
// ablations) for one window radius. The build compiles this
// file once per radius 1..7 (window sides 3..15) with -DZNCC_R=<radius>, in parallel.
#include "zncc_row.cuh"
#include "zncc_scan.cuh"
#include "zncc_mma.cuh"

#ifndef ZNCC_R
#error "compile with -DZNCC_R=<window radius 1..7>"
#endif

#define ZNCC_CAT2(a, b) a##b
#define ZNCC_CAT(a, b) ZNCC_CAT2(a, b)

namespace zncc {
cudaError_t ZNCC_CAT(launch_zncc_row_r, ZNCC_R)(const RowBatch& b, int threads, size_t smem, int mode,
                                                int dtype, cudaStream_t st) {
    return launch_zncc_row_impl<ZNCC_R>(b, threads, smem, mode, dtype, st);
}
cudaError_t ZNCC_CAT(launch_zncc_scan_r, ZNCC_R)(const ScanArgs& a, int dtype, cudaStream_t st) {
    return launch_zncc_scan_impl<ZNCC_R>(a, dtype, st);
}
cudaError_t ZNCC_CAT(launch_zncc_mma_r, ZNCC_R)(const ScanArgs& a, int dtype, cudaStream_t st) {
    return launch_zncc_mma_impl<ZNCC_R>(a, dtype, st);
}
cudaError_t ZNCC_CAT(zncc_row_occupancy_r, ZNCC_R)(int mode, int dtype, int threads, size_t smem, bool minb2,
                                                   bool single, int* bps) {
    return zncc_row_occupancy_impl<ZNCC_R>(mode, dtype, threads, smem, minb2, single, bps);
}
}  // namespace zncc
