// Shared-memory operand layouts of the tcgen05 convolution path.
//
// Both MMA operands are K-major without swizzle: a "core matrix" is 8 rows
// of 16 bytes (8 16-bit values along K) stored contiguously (128 B).
//  - A (activations): one "plane" per group of 8 channels of one cell
//    position i of a TMEM lane (P cells per lane: plane i C/8 + channel
//    group); a plane is a column of 16-byte rows, one row per lane index r
//    (cells P r .. P r + P - 1 of the padded grid), so core matrices
//    adjacent in M are 128 B apart (SBO = 128) and the two K-groups of one
//    MMA (16 channels) are one plane apart (LBO = plane stride).  Row r + s
//    of the same plane is r's address + 16 s, so the vertical tap shift of
//    one grid row (PW / P lanes) is a plain change of start address.
//  - B (weights): per K-chunk of 16, N rows: the N/8 core matrices of
//    K-group 0, then those of K-group 1 (SBO = 128, LBO = 16 N); 32 N bytes
//    per chunk.
//    Embedding layer (c_in = 1): one chunk, N = C, K = tap (9 used, 7 zero).
//    C -> C layer: the three horizontal taps stacked along N = 3 C with
//    n = j C + co for tap kx = 2 - j; 3 (C/16) chunks, chunk = ky (C/16) + h,
//    K = input channel 16 h + k.  An MMA on input cell i of a lane whose D
//    starts at column (i - 1) C then adds block j into output cell i - 1 + j
//    of the same lane; sub-ranges of j start one block (16 C bytes) later.
#pragma once
#include <stdint.h>

namespace vmc {

__host__ __device__ __forceinline__ int tc_chunk_n(int C, int l) { return l == 0 ? C : 3 * C; }
__host__ __device__ __forceinline__ int64_t tc_chunk_bytes(int C, int l) { return 32LL * tc_chunk_n(C, l); }
__host__ __device__ __forceinline__ int tc_chunks(int C, int l) { return l == 0 ? 1 : 3 * (C / 16); }
__host__ __device__ __forceinline__ int64_t tc_layer_bytes(int C, int l) { return tc_chunks(C, l) * tc_chunk_bytes(C, l); }
__host__ __device__ __forceinline__ int64_t tc_wimg_offset(int C, int l)
{
    return l == 0 ? 0 : tc_layer_bytes(C, 0) + (int64_t)(l - 1) * tc_layer_bytes(C, 1);
}
__host__ __device__ __forceinline__ int64_t tc_wimg_bytes(int C, int D) { return tc_wimg_offset(C, D + 1); }

// byte offset of element (n, k) inside one B chunk with N rows
__host__ __device__ __forceinline__ int tc_b_elem_offset(int N, int n, int k)
{
    return (k >> 3) * (16 * N) + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

}  // namespace vmc
