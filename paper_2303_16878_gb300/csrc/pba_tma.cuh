// Tensor-memory-accelerator (TMA) tile loads into shared memory, completed on
// an mbarrier, for the staged variant of the linearisation: one warp's
// bilinear taps of one 32-point step are read from a tile of the target
// frame's texels that one lane fetched with a single bulk tensor copy.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace pba {

// Staged tile of FP16 texels (16 B each): rows x columns of the target image
// around the taps of one warp step.  A step whose taps do not fit (or that
// crosses the wrap seam of a spherical image) reads its taps directly.
constexpr int kTileRows = 4;
constexpr int kTileCols = 48;
constexpr unsigned kTileBytes = kTileRows * kTileCols * 16u;
// try_wait polls of the tile's mbarrier before a warp stops staging (an error
// flag is raised and its taps are read directly from then on)
constexpr unsigned kTileSpinLimit = 1u << 24;

__device__ __forceinline__ void tma_mbar_init(uint64_t* bar, unsigned count) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
    // make the initialisation visible to the async proxy (the TMA unit)
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One lane: order this warp's earlier generic reads of the tile before the
// async-proxy write, announce the byte count and start the 3-D tile copy
// (coordinates: word in texel, column, row) of the tensor map `map`.
__device__ __forceinline__ void tma_load_tile(void* dst, uint64_t* bar, const CUtensorMap* map, int col, int row) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kTileBytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(d),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(col), "r"(row), "r"(b)
        : "memory");
}

// Poll the mbarrier's phase `parity` at most kTileSpinLimit times; true once
// the tile has arrived.
__device__ __forceinline__ bool tma_wait(uint64_t* bar, unsigned parity) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    for (unsigned spin = 0; spin < kTileSpinLimit; ++spin) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace pba
