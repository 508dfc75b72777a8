// Tiled bulk tensor copies (TMA) from global into shared memory, completed on
// an mbarrier: the stage kernel's phase 1 moves a tile's coefficient rows,
// element constants and face constants with a handful of these instead of a
// load and a store per value and thread.  Inline PTX for sm_90+ (sm_103a here).
//
// The tensor maps (CUtensorMap) are encoded on the host and live in device
// memory; every copy starts at a column that is a multiple of the tile width,
// so the innermost coordinate is 16-byte aligned.  Columns past the end of the
// tensor are filled with zeros.
#pragma once

#include <cstdint>

#include "dgm_tc.cuh"

namespace dgm {
namespace bulk {

// one arrival on `bar` that also expects `bytes` of copies to complete on it
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

// box of `tmap` at (x, y) into dst; completes `bar`'s transaction bytes
__device__ __forceinline__ void load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(tc::smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y),
           "r"(tc::smem_addr(bar))
        : "memory");
}

// box of `tmap` at (x, y, z) into dst; completes `bar`'s transaction bytes
__device__ __forceinline__ void load_3d(void* dst, const void* tmap, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(tc::smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z),
           "r"(tc::smem_addr(bar))
        : "memory");
}

}  // namespace bulk
}  // namespace dgm
