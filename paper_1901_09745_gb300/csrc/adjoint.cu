// adjoint.cu -- hand-written reverse of the PSC collide-stream step (Liu & Wu, arXiv
// 1901.09745, Eq. 1-6, 9, 12-18) for gradients of the time-averaged drag
//     J = (1/T) sum_{t<T} sum_p F_{p,x}(t)        (F_p of Eq. 14)
// with respect to every particle position X_p and the body force F, for particles that do
// not move or spin during the rollout (u_s = 0).
//
// With u_s = 0 the solid term of Eq. 12 is sum_s B_{n,s} Omega^s_i = B_n (f_-i - f^eq_-i
// - f_i) + B_n rho w_i and the per-step drag is J_t = sum_n B_n (j_x - F_x/2): both depend
// on the positions only through each cell's total weight B_n (the split B_{n,s} of Eq. 13
// drops out). Writing g_t for the stored post-collision field and p_t = S(g_t) for the
// pulled pre-collision populations, g_{t+1} = C(p_t), the reverse sweep is
//     a_t = (dC/dp)^T lambda_{t+1} + (1/T) dJ_t/dp,      lambda_t = S^T a_t,
//     dJ/dX += sum_n Lambda_n dB_n/dX,   Lambda_n = lambda.dC/dB + (1/T)(j_x - F_x/2),
//     dJ/dF += (dC/dF)^T lambda_{t+1} + (1/T) dJ_t/dF.
// dC/dp is applied exactly: the direct (diagonal + opposite) part plus the part through
// rho and u, which costs O(Q) per cell. S^T is the push along the same links (bounce-back
// links return to the own cell), a permutation, so every adjoint value is written once.
// dB_n/dX follows Eq. 9 at eps_n and Eq. 15: dB/deps = a (1 + a)/((1 - eps) + a)^2 with
// a = tau - 1/2, deps_s/dX_p = (x_n - X_p)/|x_n - X_p| on unclamped shell cells, zero
// where eps is clamped to 0 or 1 or where sum eps >= 1 (eps_n = 1, Table 1 Step 5).
//
// The forward rollout keeps a checkpoint every K steps; the reverse sweep re-runs each
// segment forward (storing its K states) and then walks it backwards.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "capi_internal.h"
#include "psc_kernels.cuh"

namespace psc {

template <class L, typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 2)
k_adjoint(const T *__restrict__ gt, const T *__restrict__ lam_in, T *__restrict__ lam_out, Geom g,
          PhysT<T> ph, Tiles tl, Parts pd, T invT, double *dJdX, double *dFpart) {
    constexpr int Q = L::Q;
    constexpr int D = L::D;
    extern __shared__ __align__(16) unsigned char smem[];
    T *srec = reinterpret_cast<T *>(smem);                 // [cap][RW]
    T *part = srec + (size_t)tl.cap * RW;                  // [kWarps][cap][D] warp partials
    __shared__ T s_dF[kWarps][3];
    __shared__ int s_wany[kWarps];

    const int tid = threadIdx.x + L::TX * (threadIdx.y + L::TY * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY, z0 = blockIdx.z * L::TZ;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool active = cell_active<L>(g, x, y, z);
    const long long tile = blockIdx.x + (long long)g.nt[0] * (blockIdx.y + (long long)g.nt[1] * blockIdx.z);
    const long long cell = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
    const long long N = g.ncell;
    const int cap = tl.cap;
    const int cnt = (pd.n > 0) ? min(tl.count[tile], cap) : 0;   // overflow is refused on the host
    const T *recs = reinterpret_cast<const T *>(tl.blocks) + tile * block_elems<T>(cap) + head_elems<T>();
    for (int w = tid; w < cnt * RW; w += kThreads) srec[w] = recs[w];

    // ---- forward quantities of this step (pull, Eq. 5); tiles one cell clear of every face
    // address their neighbours by a fixed offset (no wrap or wall tests)
    const bool interior = x0 >= 1 && x0 + L::TX < g.n[0] && y0 >= 1 && y0 + L::TY < g.n[1] &&
                          (L::D == 2 || (z0 >= 1 && z0 + L::TZ < g.n[2]));
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    T d[Q];
    pull_q<L, T>(gt, g, x, y, z, cell, interior, active, ph.sc, d);
    T drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (L::ex(i)) j[0] += L::ex(i) > 0 ? d[i] : -d[i];
        if (L::ey(i)) j[1] += L::ey(i) > 0 ? d[i] : -d[i];
        if (L::ez(i)) j[2] += L::ez(i) > 0 ? d[i] : -d[i];
    }
    const T rho = (T)1 + drho;
    const T irho = (T)1 / rho;
    const T F[3] = {ph.F[0], ph.F[1], ph.F[2]};
    const T u[3] = {(j[0] + (T)0.5 * F[0]) * irho, (j[1] + (T)0.5 * F[1]) * irho, (j[2] + (T)0.5 * F[2]) * irho};
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];

    // ---- the cell's total solid fraction and weight (Table 1, Eq. 9 at eps_n)
    const T cx = (T)threadIdx.x, cy = (T)threadIdx.y, cz = (T)threadIdx.z;
    T seps = 0;
    if (cnt > 0) {
        __syncthreads();
        for (int k = 0; k < cnt && active; ++k) {
            const T *rk = srec + k * RW;
            T dx, dy, dz;
            cand_arm<L, T>(g, cx, cy, cz, rk[R_PX], rk[R_PY], rk[R_PZ], dx, dy, dz);
            seps += shell_eps<T>(dx * dx + dy * dy + dz * dz, rk[R_R], rk[R_FR], ph.h);
        }
    }
    const T en = seps < (T)1 ? seps : (T)1;
    const T den = ((T)1 - en) + ph.tmh;
    const T B = en * ph.tmh / den;
    const T dBde = (seps > (T)0 && seps < (T)1) ? ph.tmh * ((T)1 + ph.tmh) / (den * den) : (T)0;
    const T omB = (T)1 - B;

    // ---- adjoint of the collision at this cell. Everything the transpose needs is a
    // moment of w_i lambda_i (S0, S1 = sum w lambda e, M2 = sum w lambda e e^T) or one of the
    // two products lambda.d, lambda.d_opp, because f^eq and the Guo term are quadratic in e.
    T lam[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) lam[i] = active ? lam_in[(long long)i * N + cell] : (T)0;
    T S0 = 0, S1[3] = {0, 0, 0}, Mxx = 0, Myy = 0, Mzz = 0, Mxy = 0, Mxz = 0, Myz = 0, Ld = 0, Ldo = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T wl = (T)weight<L>(i) * lam[i];
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        S0 += wl;
        if (ex) S1[0] += ex > 0 ? wl : -wl;
        if (ey) S1[1] += ey > 0 ? wl : -wl;
        if (ez) S1[2] += ez > 0 ? wl : -wl;
        if (ex) Mxx += wl;
        if (ey) Myy += wl;
        if (ez) Mzz += wl;
        if (ex && ey) Mxy += (ex == ey) ? wl : -wl;
        if (ex && ez) Mxz += (ex == ez) ? wl : -wl;
        if (ey && ez) Myz += (ey == ez) ? wl : -wl;
        Ld += lam[i] * d[i];
        Ldo += lam[i] * d[opp<L>(i)];
    }
    const T M2u[3] = {Mxx * u[0] + Mxy * u[1] + Mxz * u[2], Mxy * u[0] + Myy * u[1] + Myz * u[2],
                      Mxz * u[0] + Myz * u[1] + Mzz * u[2]};
    const T M2F[3] = {Mxx * F[0] + Mxy * F[1] + Mxz * F[2], Mxy * F[0] + Myy * F[1] + Myz * F[2],
                      Mxz * F[0] + Myz * F[1] + Mzz * F[2]};
    const T uS1 = u[0] * S1[0] + u[1] * S1[1] + u[2] * S1[2];
    const T FS1 = F[0] * S1[0] + F[1] * S1[1] + F[2] * S1[2];
    const T uMu = u[0] * M2u[0] + u[1] * M2u[1] + u[2] * M2u[2];
    const T FMu = F[0] * M2u[0] + F[1] * M2u[1] + F[2] * M2u[2];
    const T s0q = S0 * ((T)1 - (T)1.5 * uu);
    // sum_i lambda_i feq_i / rho and sum_i lambda_i feq_-i / rho
    const T Pe = s0q + (T)3 * uS1 + (T)4.5 * uMu;
    const T Po = s0q - (T)3 * uS1 + (T)4.5 * uMu;
    const T oo = omB * ph.omega;
    // through rho at fixed u: (1-B) omega feq_i/rho - B feq_-i/rho + B w_i
    const T Arho = oo * Pe - B * Po + B * S0;
    // through u at fixed rho: grad_u feq_i = rho w (3 e + 9 (e.u) e - 3 u), feq_-i with -e,
    // grad_u G_i = guo w (-3 F + 9 (e.F) e); and G_i's explicit F at fixed u
    T Au[3], dFu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T gi = (T)3 * S1[a] + (T)9 * M2u[a] - (T)3 * u[a] * S0;
        const T go = -(T)3 * S1[a] + (T)9 * M2u[a] - (T)3 * u[a] * S0;
        Au[a] = rho * (oo * gi - B * go) + omB * ph.guo * ((T)9 * M2F[a] - (T)3 * F[a] * S0);
        dFu[a] = omB * ph.guo * gi;
    }
    // dC/dB . lambda: omega (d - dfeq) + (d_-i - dfeq_-i - d_i) + (rho - 1) w_i - G_i
    const T Ldfe = drho * S0 + rho * (Pe - S0);
    const T Ldfo = drho * S0 + rho * (Po - S0);
    const T LG = ph.guo * ((T)3 * FS1 - (T)3 * uF * S0 + (T)9 * FMu);
    const T dCdB = ph.omega * (Ld - Ldfe) + (Ldo - Ldfo - Ld) + drho * S0 - LG;

    // a_k = lambda_k (1 - (1-B) omega - B) + B lambda_-k + Arho + Au.(e_k - u)/rho + (B/T) e_kx,
    // pushed back along the link it was pulled from (S^T)
    const T diag = (T)1 - oo - B;
    const NbrIdx nb = interior ? NbrIdx{} : make_nbr_idx<L>(g, x, y, z);
    const T c0 = Arho - (Au[0] * u[0] + Au[1] * u[1] + Au[2] * u[2]) * irho;
    const T Av[3] = {Au[0] * irho + invT * B, Au[1] * irho, Au[2] * irho};
    if (active) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T a = lam[k] * diag + B * lam[opp<L>(k)] + c0;
            if (L::ex(k)) a += L::ex(k) > 0 ? Av[0] : -Av[0];
            if (L::ey(k)) a += L::ey(k) > 0 ? Av[1] : -Av[1];
            if (L::ez(k)) a += L::ez(k) > 0 ? Av[2] : -Av[2];
            if (interior) {
                lam_out[(long long)k * N + cell - (L::ex(k) + L::ey(k) * sy + L::ez(k) * sz)] = a;
            } else {
                lam_out[src_index<L>(nb, k, cell, N)] = a;   // S^T: the pull's source, written once
            }
        }
    }

    // ---- body force: through u (du/dF = I/(2 rho)), explicit in G, and J_t's -B F_x/2;
    // one partial per block, accumulated over the steps without atomics
    T vF[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vF[a] = active ? (T)0.5 * Au[a] * irho + dFu[a] : (T)0;
    vF[0] -= active ? (T)0.5 * invT * B : (T)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) vF[a] += __shfl_xor_sync(kFull, vF[a], off);
    if (lane == 0) for (int a = 0; a < 3; ++a) s_dF[warp][a] = vF[a];

    // ---- positions: Lambda_n dB/deps_n deps_s/dX_s on unclamped shell cells
    const T Lam = dCdB + invT * (j[0] - (T)0.5 * F[0]);
    const T coef = (active && dBde != (T)0) ? Lam * dBde : (T)0;
    const bool wany = __any_sync(kFull, coef != (T)0);
    if (lane == 0) s_wany[warp] = wany;
    __syncthreads();
    if (tid < 3) {
        T sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += s_dF[w][tid];
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        dFpart[3 * blk + tid] += (double)sum;
    }
    if (cnt == 0) return;
    if (wany) {
        for (int k = 0; k < cnt; ++k) {
            const T *rk = srec + k * RW;
            T v[3] = {0, 0, 0};
            bool hit = false;
            if (coef != (T)0) {
                T dx, dy, dz;
                cand_arm<L, T>(g, cx, cy, cz, rk[R_PX], rk[R_PY], rk[R_PZ], dx, dy, dz);
                const T d2 = dx * dx + dy * dy + dz * dz;
                const T r = rk[R_R];
                if (d2 < (r + ph.h) * (r + ph.h)) {
                    const T dist = sqrt_t(d2);
                    const T e = rk[R_FR] - (dist - r);
                    if (dist > r - ph.h && e > (T)0 && e < (T)1 && dist > (T)0) {
                        const T c = coef / dist;
                        v[0] = c * dx; v[1] = c * dy; v[2] = c * dz;
                        hit = true;
                    }
                }
            }
            if (__any_sync(kFull, hit)) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int a = 0; a < D; ++a) v[a] += __shfl_xor_sync(kFull, v[a], off);
            }
            if (lane == 0) for (int a = 0; a < D; ++a) part[((size_t)warp * cap + k) * D + a] = v[a];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < cnt * D; idx += kThreads) {
        const int k = idx / D, a = idx - k * D;
        T sum = 0;
        for (int w = 0; w < kWarps; ++w)
            if (s_wany[w]) sum += part[((size_t)w * cap + k) * D + a];
        if (sum != (T)0) atomicAdd(&dJdX[3 * bits_id(srec[k * RW + R_ID]) + a], (double)sum);
    }
}

// dJ/dF = sum of the per-block partials
__global__ void k_sum_parts(const double *part, long long nblk, double *out) {
    __shared__ double s[3][256];
    double a[3] = {0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int c = 0; c < 3; ++c) a[c] += part[3 * b + c];
    for (int c = 0; c < 3; ++c) s[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = s[threadIdx.x][0];
}

// J += (1/T) sum_p F_{p,x} of the step just taken
__global__ void k_sum_fx(const double *F, int n, double invT, double *J) {
    __shared__ double s[256];
    double a = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) a += F[3 * p];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J += invT * s[0];
}

template <class L, typename T>
cudaError_t launch_adjoint_t(const void *gt, const void *lam_in, void *lam_out, const Geom &g, const Phys &ph,
                             const Tiles &tl, const Parts &pd, double invT, double *dJdX, double *dFpart,
                             cudaStream_t s) {
    const size_t smem = (size_t)tl.cap * RW * sizeof(T) + (size_t)kWarps * tl.cap * L::D * sizeof(T);
    auto kern = k_adjoint<L, T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.nt[0], g.nt[1], g.nt[2]);
    dim3 block(L::TX, L::TY, L::TZ);
    kern<<<grid, block, smem, s>>>((const T *)gt, (const T *)lam_in, (T *)lam_out, g, make_phys<T>(ph, L::Q), tl, pd,
                                   (T)invT, dJdX, dFpart);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(int storage, int lattice, const void *gt, const void *lam_in, void *lam_out,
                           const Geom &g, const Phys &ph, const Tiles &tl, const Parts &pd, double invT,
                           double *dJdX, double *dFpart, cudaStream_t s) {
    if (storage == ST_F64) {
        return lattice == 9 ? launch_adjoint_t<D2Q9, double>(gt, lam_in, lam_out, g, ph, tl, pd, invT, dJdX, dFpart, s)
                            : launch_adjoint_t<D3Q19, double>(gt, lam_in, lam_out, g, ph, tl, pd, invT, dJdX, dFpart, s);
    }
    return lattice == 9 ? launch_adjoint_t<D2Q9, float>(gt, lam_in, lam_out, g, ph, tl, pd, invT, dJdX, dFpart, s)
                        : launch_adjoint_t<D3Q19, float>(gt, lam_in, lam_out, g, ph, tl, pd, invT, dJdX, dFpart, s);
}

}  // namespace psc

using namespace psc;

#define ACK(call, what)                                         \
    do {                                                        \
        lbm_status st_ = ctx_cuda(ctx, (call), (what));         \
        if (st_ != LBM_OK) { status = st_; goto done; }         \
    } while (0)

// Workspace of the adjoint, kept by the context between calls: checkpoints [nseg], segment
// states [K], two adjoint fields, gradients + J, scratch forces and torques, per-block
// partials of dJ/dF.
struct AdjSpace {
    char *ckpt, *seg, *lam[2];
    double *dJX, *dJF, *dJ, *sF, *sT, *dFpart;
    size_t pop, popa, v3, need;
    long long nblk;
    int nseg;
};

static AdjSpace adj_layout(const lbm_ctx *ctx, int nsteps, int K) {
    AdjSpace a;
    const int n = ctx->np;
    a.nseg = (nsteps + K - 1) / K;
    a.pop = (size_t)ctx->g.ncell * ctx->q * ctx->elem;
    a.v3 = (size_t)(n > 0 ? n : 1) * 3 * sizeof(double);
    const size_t v3a = (a.v3 + 255) & ~(size_t)255;
    a.popa = (a.pop + 255) & ~(size_t)255;      // buffer stride, 256-byte aligned
    a.nblk = (long long)ctx->g.nt[0] * ctx->g.nt[1] * ctx->g.nt[2];
    const size_t fpa = ((size_t)a.nblk * 3 * sizeof(double) + 255) & ~(size_t)255;
    a.need = a.popa * ((size_t)a.nseg + (size_t)K + 2) + 3 * v3a + 256 + fpa;
    char *base = (char *)ctx->adj;
    a.ckpt = base;
    a.seg = a.ckpt + a.popa * (size_t)a.nseg;
    a.lam[0] = a.seg + a.popa * (size_t)K;
    a.lam[1] = a.seg + a.popa * (size_t)(K + 1);
    a.dJX = (double *)(a.lam[1] + a.popa);
    a.dJF = a.dJX + 3 * (size_t)(n > 0 ? n : 1);
    a.dJ = a.dJF + 3;
    a.sF = (double *)((char *)a.dJX + v3a + 256);
    a.sT = (double *)((char *)a.sF + v3a);
    a.dFpart = (double *)((char *)a.sT + v3a);
    return a;
}

// Forward half: T steps from the context's state with a checkpoint every K, J summed on the
// device. Leaves the checkpoints and the tile lists for lbm_adjoint_backward.
extern "C" lbm_status lbm_adjoint_forward(lbm_ctx *ctx, int nsteps, int checkpoint_every, double *J,
                                          long long *token, int on_device) {
    NvtxRange nvtx_("lbm_adjoint_forward");
    if (!ctx) return LBM_ERR_ARG;
    if (nsteps < 1 || checkpoint_every < 1) { ctx_error(ctx, "nsteps and checkpoint_every must be >= 1"); return LBM_ERR_ARG; }
    if (ctx->p.storage != LBM_F32 && ctx->p.storage != LBM_F64) {
        ctx_error(ctx, "the adjoint supports FP32 and FP64 storage");
        return LBM_ERR_UNSUPPORTED;
    }
    if (ctx->p.psc != LBM_PSC_MODIFIED) { ctx_error(ctx, "the adjoint supports the modified PSC scheme"); return LBM_ERR_UNSUPPORTED; }
    for (int a = 0; a < 3; ++a)
        if (ctx->p.bc[a] != LBM_BC_PERIODIC && ctx->p.bc[a] != LBM_BC_BOUNCEBACK) {
            ctx_error(ctx, "the adjoint supports periodic and wall axes only");
            return LBM_ERR_UNSUPPORTED;
        }
    const int n = ctx->np;
    const int K = checkpoint_every;
    lbm_status status = LBM_OK;
    ctx->adj_ready = 0;
    // static, non-moving particles only (u_s = 0)
    if (n > 0) {
        const size_t v3 = (size_t)n * 3 * sizeof(double);
        double *h = (double *)malloc(2 * v3);
        if (!h) return LBM_ERR_OOM;
        cudaError_t e = cudaMemcpyAsync(h, ctx->dU, v3, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char *)h + v3, ctx->dOm, v3, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        bool moving = false;
        for (int i = 0; i < 6 * n && e == cudaSuccess; ++i) moving |= (h[i] != 0.0);
        free(h);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "read particle velocities");
        if (moving) { ctx_error(ctx, "the adjoint is for static particles (U = Omega = 0)"); return LBM_ERR_UNSUPPORTED; }
    }
    {
        const size_t need = adj_layout(ctx, nsteps, K).need;
        if (ctx->adj_cap < need) {
            if (ctx->adj) cudaFree(ctx->adj);
            ctx->adj = NULL;
            ctx->adj_cap = 0;
            cudaError_t e = cudaMalloc(&ctx->adj, need);
            if (e != cudaSuccess) { ctx->adj = NULL; return ctx_cuda(ctx, e, "cudaMalloc(adjoint workspace)"); }
            ctx->adj_cap = need;
        }
    }
    {
        const AdjSpace w = adj_layout(ctx, nsteps, K);
        ACK(cudaMemsetAsync(w.dJX, 0, w.v3 + 4 * sizeof(double), ctx->stream), "memset gradients");
        const double invT = 1.0 / nsteps;
        for (int t = 0; t < nsteps; ++t) {
            if (t % K == 0) ACK(cudaMemcpyAsync(w.ckpt + w.popa * (size_t)(t / K), ctx->f[ctx->cur], w.pop,
                                                cudaMemcpyDeviceToDevice, ctx->stream), "checkpoint");
            lbm_status st = ctx_step_once(ctx);
            if (st != LBM_OK) { status = st; goto done; }
            if (n > 0) {
                k_sum_fx<<<1, 256, 0, ctx->stream>>>(ctx->dF, n, invT, w.dJ);
                ACK(cudaGetLastError(), "drag sum");
            }
        }
        if (n > 0) {
            int stats[4];
            ACK(cudaMemcpyAsync(stats, ctx->tile_stats, sizeof(stats), cudaMemcpyDeviceToHost, ctx->stream), "stats");
            ACK(cudaStreamSynchronize(ctx->stream), "sync");
            if (stats[0] > 0) {
                ctx_error(ctx, "the adjoint needs every tile's candidates to fit tile_cap (raise it)");
                status = LBM_ERR_UNSUPPORTED;
                goto done;
            }
        }
        if (J) ACK(cudaMemcpyAsync(J, w.dJ, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   ctx->stream), "copy J");
        ACK(cudaStreamSynchronize(ctx->stream), "sync");
    }
done:
    cudaStreamSynchronize(ctx->stream);
    if (status == LBM_OK) status = ctx_check_flags(ctx);
    if (status == LBM_OK) {
        ctx->adj_T = nsteps;
        ctx->adj_K = K;
        ctx->adj_mods = ctx->mods;
        ctx->adj_ready = 1;
        ctx->adj_token += 1;
        if (token) *token = ctx->adj_token;
    }
    return status;
}

// Backward half: the reverse sweep over the checkpoints of the last lbm_adjoint_forward.
extern "C" lbm_status lbm_adjoint_backward(lbm_ctx *ctx, long long token, double *dJdX, double *dJdF,
                                           int on_device) {
    NvtxRange nvtx_("lbm_adjoint_backward");
    if (!ctx) return LBM_ERR_ARG;
    if (!ctx->adj_ready || token != ctx->adj_token) {
        ctx_error(ctx, "no lbm_adjoint_forward with this token holds the adjoint workspace");
        return LBM_ERR_ARG;
    }
    if (ctx->mods != ctx->adj_mods) {
        ctx_error(ctx, "the particles or the body force changed since lbm_adjoint_forward");
        return LBM_ERR_ARG;
    }
    const int n = ctx->np;
    const int nsteps = ctx->adj_T, K = ctx->adj_K;
    lbm_status status = LBM_OK;
    const AdjSpace w = adj_layout(ctx, nsteps, K);
    Tiles tl;
    Parts scratch_parts;
    ACK(cudaMemsetAsync(w.dJX, 0, w.v3 + 3 * sizeof(double), ctx->stream), "memset gradients");
    ACK(cudaMemsetAsync(w.dFpart, 0, (size_t)w.nblk * 3 * sizeof(double), ctx->stream), "memset gradient partials");
    ACK(cudaMemsetAsync(w.lam[0], 0, w.pop, ctx->stream), "memset adjoint");
    {
        const double invT = 1.0 / nsteps;
        tl.count = ctx->tile_count; tl.list = ctx->tile_list; tl.cap = ctx->p.tile_cap;
        tl.stats = ctx->tile_stats; tl.blocks = ctx->tile_blocks; tl.order = ctx->tile_order;
        scratch_parts = ctx_parts(ctx);
        scratch_parts.F = w.sF;
        scratch_parts.T = w.sT;
        // segment by segment: restore the checkpoint, re-run the segment storing its states,
        // walk it back
        int cur = 0;
        for (int sidx = w.nseg - 1; sidx >= 0; --sidx) {
            const int t0 = sidx * K, t1 = (t0 + K < nsteps) ? t0 + K : nsteps;
            ACK(cudaMemcpyAsync(w.seg, w.ckpt + w.popa * (size_t)sidx, w.pop, cudaMemcpyDeviceToDevice, ctx->stream),
                "restore checkpoint");
            for (int t = t0 + 1; t < t1; ++t) {
                ACK(launch_collide_stream(ctx->p.storage, ctx->q, w.seg + w.popa * (size_t)(t - 1 - t0),
                                          w.seg + w.popa * (size_t)(t - t0), ctx->g, ctx->ph, tl, scratch_parts,
                                          ctx->flags, ctx->stream, &ctx->ov),
                    "segment recompute");
            }
            for (int t = t1 - 1; t >= t0; --t) {
                ACK(launch_adjoint(ctx->p.storage, ctx->q, w.seg + w.popa * (size_t)(t - t0), w.lam[cur], w.lam[cur ^ 1],
                                   ctx->g, ctx->ph, tl, ctx_parts(ctx), invT, w.dJX, w.dFpart, ctx->stream),
                    "adjoint kernel");
                cur ^= 1;
            }
        }
        k_sum_parts<<<1, 256, 0, ctx->stream>>>(w.dFpart, w.nblk, w.dJF);
        ACK(cudaGetLastError(), "dJ/dF sum");
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (dJdF) ACK(cudaMemcpyAsync(dJdF, w.dJF, 3 * sizeof(double), kind, ctx->stream), "copy dJ/dF");
        if (dJdX && n > 0) ACK(cudaMemcpyAsync(dJdX, w.dJX, (size_t)n * 3 * sizeof(double), kind, ctx->stream), "copy dJ/dX");
        ACK(cudaStreamSynchronize(ctx->stream), "sync");
    }
done:
    cudaStreamSynchronize(ctx->stream);
    if (status == LBM_OK) status = ctx_check_flags(ctx);
    return status;
}

extern "C" lbm_status lbm_adjoint_drag(lbm_ctx *ctx, int nsteps, int checkpoint_every, double *J,
                                       double *dJdX, double *dJdF, int on_device) {
    long long token = 0;
    lbm_status st = lbm_adjoint_forward(ctx, nsteps, checkpoint_every, J, &token, on_device);
    if (st != LBM_OK) return st;
    return lbm_adjoint_backward(ctx, token, dJdX, dJdF, on_device);
}

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_adjoint)
