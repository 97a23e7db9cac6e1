// Fused kz-plane pass of the FP32-mixed form (procedure steps 2-4 of Sec. 3
// for one k_z plane): y transform, x transform, kernel contraction with the
// energy increment, inverse x transform and inverse y transform, with the
// plane held in the shared memory of one thread-block cluster.
//
// A cluster of C CTAs owns one plane (nx * ny * 20 complex values) at a time.
// CTA r holds x-rows [r XL, (r+1) XL) (XL = nx / C) for all y while the y
// transforms run, then y-rows [r YL, (r+1) YL) for all x while the x
// transforms and the contraction run.  Between the two, chunk (r, d) (x-rows
// of r, y-rows of d) moves from CTA r to CTA d through distributed shared
// memory; both layouts put a chunk in one contiguous range of the buffer, so
// each CTA swaps chunks pairwise in place.  A partner signals "chunk read"
// on one mbarrier per partner (remote arrive) before the owner overwrites.
// The transforms are the in-place permuted ones: the forward transforms leave
// the frequencies in the order p = k1 N2 + k2 <-> k1 + N1 k2 and the inverse
// ones take that order back, so no scratch buffer is needed.
//
// The spectrum makes one HBM round trip for the whole of steps 2-4 instead of
// five (y, x, contraction, x, y passes).
#include "common.cuh"
#include "fftreg.cuh"
#include "contract.cuh"
#include "pipeline.h"
#include "tma.cuh"

namespace vdwgb {

namespace {

constexpr int PLANE_THREADS = 256;
constexpr int PLANE_MAXV = 6;         // float4 values per thread held during a chunk swap
constexpr int PLANE_MAXC = 16;        // CTAs per cluster at most

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// shared-memory layout of one CTA for a system
struct PlaneLayout {
    size_t twy, twx, kord, buf, total;
};
__host__ __device__ inline PlaneLayout plane_layout(int nx, int ny, int C, int kstride) {
    PlaneLayout L;
    size_t off = 16 + 8 * (size_t)PLANE_MAXC;          // load barrier + per-partner barriers
    L.twy = off;
    off += al16((size_t)ny * sizeof(cx<float>));
    L.twx = off;
    off += al16((size_t)nx * sizeof(cx<float>));
    L.kord = off;
    off += al16((size_t)kstride * sizeof(unsigned short));
    L.buf = off;
    off += (size_t)(nx / C) * ny * NQ * sizeof(cx<float>);
    L.total = off;
    return L;
}

__device__ __forceinline__ void mbar_arrive_remote(unsigned long long *local_bar, unsigned rank) {
    const unsigned a = dsmem_addr(local_bar, rank);
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait (~2^31 SM cycles) for a barrier completed by a remote arrive
__device__ __forceinline__ bool mbar_wait_cluster(unsigned long long *bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

// Swap chunks with every partner.  Source layout: chunk d holds records
// (a * B + b) for a < A, b < B (a runs over the partner's rows); destination:
// (b * A + a).  to_x: from the y layout (a = y-row, b = x-row) to the x
// layout, else back.  Chunks are CH = A * B * 20 complex values.
__device__ __noinline__ bool swap_chunks(cx<float> *buf, int C, unsigned rank, int A, int B,
                                            unsigned long long *pbar, unsigned parity) {
    const int CH = A * B * NQ;
    const int CH4 = CH / 2;                       // float4 units
    bool ok = true;
    for (int r = 0; r < C; ++r) {
        const unsigned d = rank ^ (unsigned)r;
        float4 v[PLANE_MAXV];
        const unsigned src = dsmem_addr(buf + (size_t)rank * CH, d);
#pragma unroll
        for (int k = 0; k < PLANE_MAXV; ++k) {
            const int e = threadIdx.x + k * PLANE_THREADS;
            if (e < CH4) v[k] = dsmem_ld4(src + 16u * (unsigned)e);
        }
        __syncthreads();                          // this CTA has read chunk `rank` of d
        if (r == 0) {
            // own chunk: read by this CTA only
        } else {
            if (threadIdx.x == 0) mbar_arrive_remote(&pbar[rank], d);
            // d must have read chunk d of this CTA before it is overwritten
            if (!mbar_wait_cluster(&pbar[d], parity)) ok = false;
        }
        cx<float> *dst = buf + (size_t)d * CH;
#pragma unroll
        for (int k = 0; k < PLANE_MAXV; ++k) {
            const int e = threadIdx.x + k * PLANE_THREADS;
            if (e < CH4) {
                const int rec = e / 10, q = e - rec * 10;
                const int a = rec / B, b = rec - a * B;
                *reinterpret_cast<float4 *>(dst + ((size_t)b * A + a) * NQ + 2 * q) = v[k];
            }
        }
    }
    __syncthreads();
    return ok;
}

// Contraction of this CTA's k-points of one plane (kord order): F = phi(|k|) theta
// written over theta; returns this thread's share of sum_k sum_a Re(theta* F).
__device__ __noinline__ double contract_plane(cx<float> *buf, const unsigned short *kord, int npts, int YL, int ybase,
                                              int nx, int ny, int n1x, int n1y, float fz, float czv,
                                              float4 g012, float4 g345, const float4 *__restrict__ tab) {
    const float inv_dk = (float)(RMAX / (2.0 * 3.14159265358979323846));
    const int n2x = nx / n1x, n2y = ny / n1y;
    double eacc = 0.0;
    for (int i = threadIdx.x; i < npts; i += PLANE_THREADS) {
        const int li = kord[i];
        const int px = li / YL, yl = li - px * YL;
        const int x = fft_perm_freq(px, n1x, n2x);
        const int y = fft_perm_freq(ybase + yl, n1y, n2y);
        const int mx = x <= (nx - 1) / 2 ? x : x - nx, my = y <= (ny - 1) / 2 ? y : y - ny;
        const bool nyq_x = (nx % 2 == 0) && (x == nx / 2);
        const bool nyq_y = (ny % 2 == 0) && (y == ny / 2);
        const float fx = (float)mx, fy = (float)my;
        const float cxv = nyq_x ? 0.f : fx, cyv = nyq_y ? 0.f : fy;
        float k2 = g012.x * fx * fx + g012.y * fy * fy + g012.z * fz * fz +
                   2.f * (g345.x * cxv * cyv + g345.y * cxv * czv + g345.z * cyv * czv);
        k2 = k2 > 0.f ? k2 : 0.f;
        const float xk = sqrtf(k2) * inv_dk;
        const int j = (int)xk;
        const float tt = xk - (float)j;
        float4 *v4 = reinterpret_cast<float4 *>(buf + (size_t)li * NQ);
        f2_t th[NQ], F[NQ];
        load_rec_f2(v4, th);
#pragma unroll
        for (int a = 0; a < NQ; ++a) F[a] = 0ull;
        if (j < NK - 1) contract_row<true>(tab + (size_t)j * NPAIR, tt, th, F);
        eacc += (double)energy_f2(th, F);
        store_rec_f2(v4, F);
    }
    return eacc;
}

}  // namespace

// One cluster per plane at a time; planes of all fused systems form one list.
__global__ void __launch_bounds__(PLANE_THREADS, 2)
    k_plane(const SysDev *__restrict__ sys, const int *__restrict__ prefix, int nsys, int total,
            const float4 *__restrict__ tab, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[PLANE_THREADS / 32];
    unsigned long long *lbar = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *pbar = reinterpret_cast<unsigned long long *>(smem + 16);
    const unsigned rank = cluster_rank();
    if (threadIdx.x == 0) {
        mbar_init(lbar, 1);
        for (int i = 0; i < PLANE_MAXC; ++i) mbar_init(&pbar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    cluster_sync();                               // every CTA's barriers initialised
    unsigned lph = 0u, xph = 0u;
    bool failed = false;
    int cur_sys = -1;
    for (int t = (int)cluster_index(); t < total; t += (int)cluster_count()) {
        const int si = find_sys(prefix, nsys, t);
        const SysDev &S = sys[si];
        const int kz = t - prefix[si];
        const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh, C = S.fused;
        const int XL = nx / C, YL = ny / C;
        const PlaneLayout PL = plane_layout(nx, ny, C, S.kstride);
        cx<float> *twy = reinterpret_cast<cx<float> *>(smem + PL.twy);
        cx<float> *twx = reinterpret_cast<cx<float> *>(smem + PL.twx);
        unsigned short *kord = reinterpret_cast<unsigned short *>(smem + PL.kord);
        cx<float> *buf = reinterpret_cast<cx<float> *>(smem + PL.buf);
        cx<float> *spec = reinterpret_cast<cx<float> *>(S.spec);
        const int x0 = (int)rank * XL;
        // ---- load this CTA's x-rows of the plane: record (y, xl) at (y XL + xl)
        if (threadIdx.x < 32 && !failed) {
            const int lane = threadIdx.x;
            const unsigned kb = (unsigned)(S.kstride * sizeof(unsigned short));
            fence_proxy_async();
            if (lane == 0) mbar_expect_tx(lbar, (unsigned)(XL * ny) * 160u + kb);
            __syncwarp();
            int y = lane / XL, xl = lane - (lane / XL) * XL;
            const int dy = 32 / XL, dx = 32 - dy * XL;
            for (int rr = lane; rr < XL * ny; rr += 32) {
                bulk_g2s(buf + (size_t)rr * NQ, spec + (((size_t)(x0 + xl) * ny + y) * nzh + kz) * NQ, 160u, lbar);
                xl += dx;
                y += dy;
                if (xl >= XL) {
                    xl -= XL;
                    ++y;
                }
            }
            if (lane == 0) bulk_g2s(kord, S.kord + ((size_t)kz * C + rank) * S.kstride, kb, lbar);
        }
        if (si != cur_sys) {
            const cx<float> *gy = reinterpret_cast<const cx<float> *>(S.tw[1]);
            const cx<float> *gx = reinterpret_cast<const cx<float> *>(S.tw[0]);
            for (int i = threadIdx.x; i < ny; i += PLANE_THREADS) twy[i] = gy[i];
            for (int i = threadIdx.x; i < nx; i += PLANE_THREADS) twx[i] = gx[i];
            cur_sys = si;
        }
        if (!failed) {
            bool ok = mbar_wait(lbar, lph);
            if (!ok) {
                atomicExch(err, 1);
                ok = mbar_wait(lbar, lph);       // let copies in flight land before going on
            }
            failed = !__syncthreads_or(!ok) ? failed : true;
        }
        lph ^= 1u;
        __syncthreads();
        // ---- y transforms: lines (xl, a), element y; stride XL 20
        fft_ip_auto<false>(buf, ny, XL * NQ, XL * NQ, twy);
        cluster_sync();                           // partners' y transforms done
        if (!swap_chunks(buf, C, rank, YL, XL, pbar, xph)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
        }
        xph ^= 1u;
        // ---- x transforms: records (x, yl) at (x YL + yl); lines (yl, a), element x
        fft_ip_auto<false>(buf, nx, YL * NQ, YL * NQ, twx);
        // ---- contraction at the k-points (x, y0 + yl) of this plane in table order
        double eacc = 0.0;
        {
            const bool nyq_z = (nz % 2 == 0) && (kz == nz / 2);
            const int mz = nyq_z ? -kz : kz;
            const float4 g012 = make_float4((float)S.g[0], (float)S.g[1], (float)S.g[2], 0.f);
            const float4 g345 = make_float4((float)S.g[3], (float)S.g[4], (float)S.g[5], 0.f);
            eacc = contract_plane(buf, kord, nx * YL, YL, (int)rank * YL, nx, ny, S.sx1, S.sy1, (float)mz,
                                  nyq_z ? 0.f : (float)mz, g012, g345, tab);
            // energy partial of (plane, rank); half-spectrum weight 2 except k_z = 0 and Nyquist
            const double w = (kz == 0 || nyq_z) ? 1.0 : 2.0;
            for (int o = 16; o > 0; o >>= 1) eacc += __shfl_down_sync(0xffffffffu, eacc, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = eacc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int i = 0; i < PLANE_THREADS / 32; ++i) s += red[i];
                S.epart[(size_t)kz * C + rank] = w * s;
            }
        }
        __syncthreads();
        fft_ip_auto<true>(buf, nx, YL * NQ, YL * NQ, twx);
        cluster_sync();                           // partners' inverse x transforms done
        if (!swap_chunks(buf, C, rank, XL, YL, pbar, xph)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
        }
        xph ^= 1u;
        fft_ip_auto<true>(buf, ny, XL * NQ, XL * NQ, twy);
        // ---- store the x-rows back: record (y, xl) -> (x0 + xl, y, kz); 16-byte vectors
        {
            const int n4 = XL * ny * 10;
            for (int e = threadIdx.x; e < n4; e += PLANE_THREADS) {
                const int rec = e / 10, q = e - rec * 10;
                const int y = rec / XL, xl = rec - y * XL;
                const float4 v = *reinterpret_cast<const float4 *>(buf + (size_t)rec * NQ + 2 * q);
                *reinterpret_cast<float4 *>(spec + (((size_t)(x0 + xl) * ny + y) * nzh + kz) * NQ + 2 * q) = v;
            }
        }
        fence_proxy_async();                      // generic reads of buf before the next bulk writes
        __syncthreads();
    }
    cluster_sync();                               // no CTA leaves while partners may touch its memory
    if (threadIdx.x == 0) {
        mbar_inval(lbar);
        for (int i = 0; i < PLANE_MAXC; ++i) mbar_inval(&pbar[i]);
    }
}

size_t plane_smem(int nx, int ny, int C) {
    const int kstride = ((nx * (ny / C)) + 7) & ~7;
    return plane_layout(nx, ny, C, kstride).total;
}

cudaError_t init_plane_kernel(size_t maxsmem) {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_plane, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(maxsmem - sizeof(double) * (PLANE_THREADS / 32)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_plane, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_plane, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

int plane_max_clusters(int C, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void *)k_plane, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_plane(const LaunchSet &ls, cudaStream_t st) {
    if (ls.total[5] == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ls.grid[5] * ls.cluster), 1, 1);
    cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
    cfg.dynamicSmemBytes = ls.smem[5];
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ls.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_plane, ls.sys, ls.prefix[5], ls.nsys, ls.total[5],
                              reinterpret_cast<const float4 *>(ls.table), ls.err);
}

}  // namespace vdwgb

