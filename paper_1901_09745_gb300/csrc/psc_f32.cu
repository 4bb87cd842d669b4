// psc_f32.cu -- instantiates the PSC step kernels for populations stored as float.
// (One translation unit per storage type so the library builds in parallel.)
#include "psc_kernels.cuh"

namespace psc {

cudaError_t launch_collide_stream_f32(int lattice, const void *fin, void *fout, const Geom &g,
                                    const Phys &ph, const Tiles &tl, const Parts &pd, int *flags,
                                    cudaStream_t s, Overlap *ov) {
    return launch_collide_stream_storage<float>(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
}

cudaError_t launch_gather_f32(int lattice, const void *fin, double *f_out, double *rho, double *u,
                            const Geom &g, const Phys &ph, cudaStream_t s) {
    return launch_gather_storage<float>(lattice, fin, f_out, rho, u, g, ph, s);
}

cudaError_t launch_set_f32(int lattice, const double *f, void *fout, const Geom &g, const Phys &ph,
                         cudaStream_t s) {
    return launch_set_storage<float>(lattice, f, fout, g, ph, s);
}

}  // namespace psc

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_psc_f32)
