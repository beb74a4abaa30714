// kernels.h -- argument blocks and launchers of the device kernels (internal to libzncc).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace zncc {

enum { kModeRaw = 0, kModeHPair = 1, kModeWta = 2 };   // k_zncc_row variants
enum { kLineStore = 0, kLineWta = 1 };                  // k_line_pair variants

struct RowArgs {
    const uint8_t* left;
    const uint8_t* right;
    int pitch, W, H, D;
    const int* SL;            // [H][W]           window sums of the left image
    const float* ISL;         // [H][W]           1/sigma of the left image
    const int* SR;            // [H][W+D-1]       right image, centre c at column c+D-1
    const float* ISR;
    int nch, ds;              // chunks per row (ceil(W/16)) and disparities per block
    int d_begin, d_end;       // disparity range of this launch
    void* vol;                // output [H][W][dstride] of float or half
    long long dstride;        // elements per pixel in the output
    int d_out0;               // disparity stored at index 0 of a pixel's entries
    int vec;                  // 16-byte (float) / 8-byte (half) accesses allowed
    const float* eh;          // [H][W] horizontal edge weights (HPair mode)
    float s;                  // 1 - K
    unsigned long long* keys; // [H][W] WTA keys (Wta mode)
};

struct LineArgs {
    void* vol;                // float or half cost volume
    long long elem_stride;    // elements between consecutive positions of a line
    long long line_stride;    // elements between consecutive lines
    int n, nlines;            // line length, number of lines
    int dcount;               // valid disparities per pixel entry (<= elements per pixel)
    int ds, lpc, nch;         // disparities per block, lines per block, chunks per line
    const float* ew;          // edge weights: ew[line * ew_line_stride + pos]
    long long ew_line_stride;
    float s;
    int vec;
    unsigned long long* keys; // WTA: key of pixel line*pix_line + pos*pix_pos
    long long pix_line, pix_pos;
    int d_base;               // disparity of local index 0 (WTA)
};

size_t zncc_row_smem_bytes(int R, int mode, int nch, int ds);
size_t line_pair_smem_bytes(int lpc, int nch, int ds);

cudaError_t launch_zncc_row(int R, const RowArgs& a, int mode, int dtype, cudaStream_t st);
cudaError_t launch_line_pair(const LineArgs& a, int mode, int dtype, cudaStream_t st);
cudaError_t launch_window_stats(const uint8_t* img, int pitch, int W, int H, int r, int x_begin,
                                int nx, int* S, int* Q, float* isig, cudaStream_t st);
cudaError_t launch_dt_weights(const uint8_t* guide, int pitch, int W, int H, float K,
                              float inv_sr255, float* eh, float* evt, cudaStream_t st);
cudaError_t launch_wta_volume(const void* cost, int dtype, int W, int H, int D, uint16_t* disp,
                              cudaStream_t st);
cudaError_t launch_wta_finalize(const unsigned long long* keys, int npix, uint16_t* disp,
                                cudaStream_t st);

// per-radius launchers, one translation unit each
#define ZNCC_DECLARE_ROW(R) \
    cudaError_t launch_zncc_row_r##R(const RowArgs& a, int mode, int dtype, cudaStream_t st);
ZNCC_DECLARE_ROW(1)
ZNCC_DECLARE_ROW(2)
ZNCC_DECLARE_ROW(3)
ZNCC_DECLARE_ROW(4)
ZNCC_DECLARE_ROW(5)
ZNCC_DECLARE_ROW(6)
ZNCC_DECLARE_ROW(7)
#undef ZNCC_DECLARE_ROW

}  // namespace zncc
