// The encoder's prepared scene (Sec. 3.3-3.4): the rows kept by the prune in (Morton code,
// original index) order, the octree, the duplicate counts and the quantized attributes.
// Filled on the host (encode.cu, `prepare`) or on the device (k_prepare.cu,
// `prepare_device`), with identical contents.
#pragma once
#include <stdint.h>

#include <vector>

#include "sgs_internal.h"

namespace sgs {

struct Prepared {
    uint32_t depth = 0, n_in = 0;
    std::vector<uint32_t> keep;          // row -> original index
    std::vector<uint64_t> leaves;        // unique Morton codes
    std::vector<uint32_t> dups;          // {rank, extra} pairs
    std::vector<std::vector<uint8_t>> levels;
    uint32_t bits[kNChan];
    std::vector<uint8_t> q8;             // [rows][56] when every width <= 8
    std::vector<uint16_t> q16;           // [rows][56]
    std::vector<uint32_t> coord;         // [3][rows] voxel coordinates of the rows
    float step[kNChan], offset[kNChan];
    uint32_t rows() const { return (uint32_t)keep.size(); }
};

// Device preparation on `device`: the host `prepare`'s results exactly.  SGS_E_INVALID for
// the inputs `prepare` refuses, SGS_E_NOMEM, SGS_E_CUDA.
int prepare_device(int device, const float *pos, const float *attr, uint32_t n, uint32_t D, const uint32_t *bits,
                   Prepared &P);

}  // namespace sgs
