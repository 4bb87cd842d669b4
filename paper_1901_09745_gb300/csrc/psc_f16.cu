// psc_f16.cu -- instantiates the PSC step kernels for populations stored as __half.
// (One translation unit per storage type so the library builds in parallel.)
#include "psc_kernels.cuh"

namespace psc {

cudaError_t launch_collide_stream_f16(int lattice, const void *fin, void *fout, const Geom &g,
                                    const Phys &ph, const Tiles &tl, const Parts &pd, int *flags,
                                    cudaStream_t s, Overlap *ov) {
    return launch_collide_stream_storage<__half>(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
}

cudaError_t launch_gather_f16(int lattice, const void *fin, double *f_out, double *rho, double *u,
                            const Geom &g, const Phys &ph, cudaStream_t s) {
    return launch_gather_storage<__half>(lattice, fin, f_out, rho, u, g, ph, s);
}

cudaError_t launch_set_f16(int lattice, const double *f, void *fout, const Geom &g, const Phys &ph,
                         cudaStream_t s) {
    return launch_set_storage<__half>(lattice, f, fout, g, ph, s);
}

}  // namespace psc

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_psc_f16)
