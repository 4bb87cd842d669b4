// tma.cuh -- the tensor-memory-accelerator (TMA) staging of the pull streaming (Eq. 1).
//
// For a lattice tile with origin (x0, y0, z0), the pull of direction i reads the previous
// step's values at the cells x - e_i of the tile: one box of TZ x TY rows of the tile's
// shape, shifted by -e_i, in the population plane i. One elected thread issues one TMA
// tiled copy (cp.async.bulk.tensor) per direction into a shared-memory stage, all of them
// completing on one mbarrier; the block's warps then read their cells' values from shared
// memory. The copies of the next tile are in flight while the block computes the current
// one, so the bytes in flight per SM no longer depend on registers or resident warps.
//
// Box geometry: the TMA rule that a copy's innermost coordinate times the element size is
// a multiple of 16 bytes holds because every box starts at x0 (a multiple of 32) or, for
// e_x = +1, at x0 - AL (AL = 16 bytes in elements); the box is TX + AL elements wide, which
// covers x0 - 1 .. x0 + TX - 1 (e_x = +1) and x0 + 1 .. x0 + TX (e_x = -1). Rows of the box
// follow the tile's rows shifted by -e_y and -e_z. Out-of-range parts of a box (beyond a
// face of the lattice) are filled with zeros by the TMA unit and are never read: cells on a
// face of the lattice take their values from global memory (periodic wrap, bounce-back).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace psc {

template <class L, typename S>
struct TmaBox {
    static constexpr int AL = 16 / (int)sizeof(S);       // 16 bytes in elements
    static constexpr int BX = L::TX + AL;                 // box width (elements)
    static constexpr int ROWS = L::TY * L::TZ;            // rows of a tile
    static constexpr int ELEMS = BX * ROWS;               // elements of one direction's box
    static constexpr int BYTES = ELEMS * (int)sizeof(S);
    static constexpr int STAGE_BYTES = BYTES * L::Q;      // one tile, all directions
    static_assert(BYTES % 128 == 0, "each direction's box starts on a 128-byte boundary");
    // column of the box holding the pulled value of tile column xl in direction i
    __host__ __device__ static constexpr int col(const int ex, const int xl) {
        return xl + (ex == 1 ? AL - 1 : (ex == -1 ? 1 : 0));
    }
    // x start of direction i's box relative to the tile origin
    __host__ __device__ static constexpr int xshift(const int ex) { return ex == 1 ? -AL : 0; }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive (one thread) and announce the bytes the pending copies will deliver.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete, for at most about two seconds;
// returns false if it did not (the caller records the error and stops using the stage).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return true;
}

// One tiled copy of a box into shared memory, completing on `bar`. The tensor map is a
// __grid_constant__ kernel parameter (its address is passed as a generic address).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2),
        "r"(c3)
        : "memory");
}

// Issue the copies of one tile (all directions) into `stage` (one thread).
template <class L, typename S>
__device__ __forceinline__ void tma_issue_tile(const CUtensorMap *map, unsigned char *stage, uint64_t *bar, int x0,
                                               int y0, int z0) {
    using B = TmaBox<L, S>;
    mbar_expect_tx(bar, (unsigned)B::STAGE_BYTES);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        unsigned char *dst = stage + (size_t)i * B::BYTES;
        const int cx = x0 + B::xshift(L::ex(i)), cy = y0 - L::ey(i);
        if (L::D == 2) tma_load_3d(dst, map, bar, cx, cy, i);
        else tma_load_4d(dst, map, bar, cx, cy, z0 - L::ez(i), i);
    }
}

}  // namespace psc
