// Dense passes of the sweep on HBM-resident tensors (dense.cu): the kernel
// arguments and the host entry shared by the pass call of the C ABI and the
// wide sampler.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace pw {

struct DenseArgs {
    float2* L;             // ntens tensors of 2^W complex entries, updated in place
    const float2* ops;     // ntens operators of 2^k x 2^k entries, Op[t'][t] at t' * 2^k + t
    const float2* diag;    // per tensor diag_stride entries: ndiag tables of 32
    int diag_stride;
    uint64_t ntens;
    uint64_t stride;       // entries from one tensor to the next (>= 2^W)
    int W, k;
    int swz;               // 1: entry i stored at i ^ ((i >> 4) & 15)
    int tile_pos[8];       // operator index bit j <-> tensor index bit tile_pos[j]
    int row_pos[7];        // the index bits numbering the 128 rows of a GEMM tile
    int outer_pos[32];     // the index bits numbering the tiles of a tensor (the other bits are
                           // fixed to 0 in the tiles processed)
    int nouter;
    int ndiag;
    int diag_nb[4];
    int diag_pos[4][5];
    int* err;              // device flag: a bounded wait ran out
    // set by dense_run (any order of the row bits above is accepted and
    // replaced): the GEMM's column bit j is operator index bit col_of[j], and
    // the producers' entry order takes tensor index bit e_bits[i] as bit i
    int col_of[8];
    int e_bits[13];
};

// Enqueue one pass on stream st; t0 / t1 (nullable) are recorded right
// before and after the GEMM kernel.
int dense_run(int gemm, const DenseArgs& a, cudaStream_t st, cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);

}  // namespace pw
