// psc_bin.cu -- particle binning into lattice-tile candidate lists, and f(r) per particle.
//
// Table 1 of the paper loops over particles and, for each, over the cells of its bounding
// box. On the GPU the loop is inverted: each particle inserts itself into every lattice
// tile that its (r + h)-widened bounding box meets, so the fused collide-stream kernel can
// hold the tile's few candidates in shared memory and evaluate every cell against them.
#include <math.h>

#include "psc_kernels.cuh"

namespace psc {

constexpr int kBinBatch = 8;   // tiles whose slot atomics one thread has in flight at once

__global__ void k_bin(int dim, Geom g, double h, Tiles tl, Parts pd) {
    pdl_launch();     // the packing kernel may start; it waits for this one to finish
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int mx = 0;   // largest slot taken by this thread
    if (p < pd.n) {
        for (int c = 0; c < 3; ++c) { pd.F[3 * p + c] = 0.0; pd.T[3 * p + c] = 0.0; }
        if (pd.Pf) {   // FP32 record data, converted once per particle
            pd.Pf[2 * p] = make_float4((float)pd.R[p], (float)pd.Fr[p], (float)pd.U[3 * p], (float)pd.U[3 * p + 1]);
            pd.Pf[2 * p + 1] = make_float4((float)pd.U[3 * p + 2], (float)pd.Om[3 * p], (float)pd.Om[3 * p + 1],
                                           (float)pd.Om[3 * p + 2]);
        }
        int ra[3][2], rb[3][2], nr[3], len[3];
        const double r = pd.R[p];
        // a tile is a candidate only if some cell centre of it can lie within r + h (the
        // distance from the particle to the tile's box of cell centres; a margin far above
        // the FP32 rounding of these distances keeps the test conservative)
        const float reach = (float)(r + h) + 0.01f;
        // the centre wrapped into [0, n] on periodic axes: the culling below compares it with
        // its images at +-n only, and callers may pass positions any number of periods out
        double xw[3] = {pd.X[3 * p], pd.X[3 * p + 1], dim == 3 ? pd.X[3 * p + 2] : 0.0};
        for (int ax = 0; ax < dim; ++ax)
            if (g.periodic[ax]) xw[ax] = wrap_centre(xw[ax], g.n[ax], g.inv_n[ax]);
        const float xp[3] = {(float)xw[0], (float)xw[1], (float)xw[2]};
        for (int ax = 0; ax < 3; ++ax) {
            if (ax >= dim) { nr[ax] = 1; ra[ax][0] = rb[ax][0] = 0; len[ax] = 1; continue; }
            const double X = xw[ax];
            const int lo = (int)ceil(X - r - h), hi = (int)floor(X + r + h);
            nr[ax] = axis_tile_ranges(lo, hi, g.n[ax], tile_ext(dim, ax), g.nt[ax], g.periodic[ax], ra[ax], rb[ax]);
            len[ax] = 0;
            for (int k = 0; k < nr[ax]; ++k) len[ax] += rb[ax][k] - ra[ax][k] + 1;
        }
        // every tile of the box, kBinBatch at a time: the slot atomics of a batch are
        // independent, so their round trips overlap
        const int total = len[0] * len[1] * len[2];
        for (int k0 = 0; k0 < total; k0 += kBinBatch) {
            long long tile[kBinBatch];
            int slot[kBinBatch];
#pragma unroll
            for (int q = 0; q < kBinBatch; ++q) {
                const int k = k0 + q;
                if (k < total) {
                    const int kx = k % len[0], kyz = k / len[0];
                    const int tx = axis_tile(kx, nr[0], ra[0], rb[0]);
                    const int ty = axis_tile(kyz % len[1], nr[1], ra[1], rb[1]);
                    const int tz = axis_tile(kyz / len[1], nr[2], ra[2], rb[2]);
                    tile[q] = -1;
                    const int org[3] = {tx * tile_ext(dim, 0), ty * tile_ext(dim, 1), tz * tile_ext(dim, 2)};
                    const int ext[3] = {tile_ext(dim, 0), tile_ext(dim, 1), tile_ext(dim, 2)};
                    if (tile_in_reach(xp, reach, org, ext, g.n, g.periodic, dim)) {
                        tile[q] = PSC_IDX(tx + (long long)g.nt[0] * (ty + (long long)g.nt[1] * tz),
                                          (long long)g.nt[0] * g.nt[1] * g.nt[2], CHK_TILE);
                        slot[q] = atomicAdd(&tl.count[tile[q]], 1);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kBinBatch; ++q) {
                if (k0 + q < total && tile[q] >= 0) {
                    if (slot[q] < tl.cap) tl.list[tile[q] * tl.cap + slot[q]] = p;
                    else if (slot[q] == tl.cap) atomicAdd(&tl.stats[0], 1);
                    mx = max(mx, slot[q] + 1);
                }
            }
        }
    }
    // the largest count: one atomic per warp, not per (particle, tile)
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&tl.stats[1], mx);
}

// Eq. 18 with V_a of Eq. 17 (3D) or Eq. 19 (2D), the integrand read as the sphere (disc)
// height sqrt(r^2 - x^2 - y^2) over the unit square (segment); principal arctangents.
__device__ __forceinline__ double f_of_r(int dim, double r) {
    const double r2 = r * r;
    double va;
    if (dim == 2) {
        const double s = sqrt(r2 - 0.25);
        va = 0.5 * s + r2 * atan(0.5 / s);
    } else {
        const double s = sqrt(r2 - 0.5);
        va = (1.0 / 12.0 - r2) * atan(0.5 * s / (0.5 - r2)) + s / 3.0 +
             (r2 - 1.0 / 12.0) * atan(0.5 / s) - (4.0 / 3.0) * r2 * r * atan(0.25 / (r * s));
    }
    return va - r + 0.5;
}

__global__ void k_f_of_r(int dim, const double *R, double *Fr, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    Fr[p] = f_of_r(dim, R[p]);
}

// One thread per particle. Sources and destinations may be the same arrays (each thread
// reads its elements before writing them), so no pointer is declared restrict.
__global__ void k_upload(Upload u) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= u.n) return;
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long k = 3LL * p + a;
        x[a] = u.X[k];
        const double v = u.U[k], o = u.Om[k];
        u.dX[k] = x[a];
        u.dU[k] = v;
        u.dOm[k] = o;
        u.dF[k] = 0.0;
        u.dT[k] = 0.0;
    }
    const double r = u.R[p];
    u.dR[p] = r;
    u.dFr[p] = f_of_r(u.dim, r);
    if (u.ref) {
        const double xr[3] = {u.ref[3LL * p], u.ref[3LL * p + 1], u.ref[3LL * p + 2]};
        if (psc::moved2(x, xr, u.n_lat, u.periodic, u.dim) > u.lim2) *u.req = 1;
    }
}

// F, T and the flag words to the caller's memory (device memory or mapped page-locked host
// memory), one thread per element.
__global__ void k_download(const double *F, const double *T, double *Fo, double *To, long long m, const int *flags,
                           int *flags_out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) {
        if (Fo) Fo[k] = F[k];
        if (To) To[k] = T[k];
    }
    if (k < 4) flags_out[k] = flags[k];
}

cudaError_t launch_bin(int dim, const Geom &g, const Phys &ph, const Tiles &tl, const Parts &pd,
                       cudaStream_t s) {
    if (pd.n <= 0) return cudaSuccess;
    const int threads = 128;
    return launch_pdl(k_bin, dim3((pd.n + threads - 1) / threads), dim3(threads), 0, s, dim, g, ph.shell_h, tl, pd);
}

long long pack_block_bytes(int rec_double, int cap) {
    return rec_double ? block_elems<double>(cap) * (long long)sizeof(double)
                      : block_elems<float>(cap) * (long long)sizeof(float);
}

cudaError_t launch_pack(int lattice, int rec_double, const Geom &g, const Tiles &tl, const Parts &pd,
                        long long ntiles, cudaStream_t s) {
    const dim3 blocks((unsigned)((g.nt[0] + kWarps - 1) / kWarps), (unsigned)g.nt[1], (unsigned)g.nt[2]);
    if (lattice == 9) {
        return rec_double ? launch_pdl(k_pack_tiles<D2Q9, double>, blocks, dim3(kThreads), 0, s, g, tl, pd, ntiles)
                          : launch_pdl(k_pack_tiles<D2Q9, float>, blocks, dim3(kThreads), 0, s, g, tl, pd, ntiles);
    }
    return rec_double ? launch_pdl(k_pack_tiles<D3Q19, double>, blocks, dim3(kThreads), 0, s, g, tl, pd, ntiles)
                      : launch_pdl(k_pack_tiles<D3Q19, float>, blocks, dim3(kThreads), 0, s, g, tl, pd, ntiles);
}

cudaError_t launch_f_of_r(int dim, const double *R, double *Fr, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    k_f_of_r<<<(n + threads - 1) / threads, threads, 0, s>>>(dim, R, Fr, n);
    return cudaGetLastError();
}

cudaError_t launch_upload(const Upload &u, cudaStream_t s) {
    if (u.n <= 0) return cudaSuccess;
    const int threads = 128;
    k_upload<<<(u.n + threads - 1) / threads, threads, 0, s>>>(u);
    return cudaGetLastError();
}

cudaError_t launch_download(const double *F, const double *T, double *Fo, double *To, long long m,
                            const int *flags, int *flags_out, cudaStream_t s) {
    const int threads = 256;
    const long long work = m > 4 ? m : 4;
    k_download<<<(unsigned)((work + threads - 1) / threads), threads, 0, s>>>(F, T, Fo, To, m, flags, flags_out);
    return cudaGetLastError();
}

}  // namespace psc

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_psc_bin)
