// Host-visible interface of the stage kernels (pipeline.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace vdwgb {

// Everything one launch of the five stages needs: device descriptors of all
// systems, per-stage tile prefix sums (device), grid and shared memory.
// Tile kinds: 0 z-forward, 1 y (both directions), 2 x (both directions),
// 3 z-inverse, 4 contraction chunks, 5 kz-planes (fused plane kernel).
struct LaunchSet {
    const SysDev *sys;       // device array [nsys]
    const int *prefix[6];    // device arrays [nsys + 1]
    int nsys;
    int total[6];            // tiles per kind over all systems
    int grid[6];
    size_t smem[6];
    int maxspan;             // contraction: kernel-table intervals staged per chunk
    const void *table;       // kernel polynomial table (float4 or dvec4), [210][NK-1]
    int twmax[6];            // longest axis of the stage over all systems (twiddle slots)
    int bufelems[6];         // complex elements of one row-tile buffer (x / y stages)
    int nbuf[6];             // x / y stages: input buffers in the ring (1..XY_MAXIN)
    int work[6];             // per kind: 1 if some system needs the scratch buffer (z, y, x, z inverse)
    int recelems;            // z-inverse: point records per staged tile
    int abelems;             // z-inverse: complex elements of one transform buffer
    int *err;                // device flag set by a stage whose bounded wait ran out
    int cluster;             // plane kernel: CTAs per cluster
};

// Row stride (complex elements) of the z-pass transform buffers for nl lines
// (10 complex lines each); odd, so that consecutive rows start in different banks.
__host__ __device__ inline int z_ld(int nl) { return 10 * nl + 1; }

// contraction chunks: at most CHUNK k-points spanning at most SPAN table
// intervals (FP32-mixed: one k-point per consumer thread)
constexpr int C32_CWARPS = 11;  // FP32 contraction: consumer warps per block (one energy partial each per chunk)
constexpr int CHUNK32 = 32 * C32_CWARPS, SPAN32 = 8, CHUNK64 = 256, SPAN64 = 8;

// Shared memory of an x / y pass block: barriers and twiddles, then nbuf
// row-tile buffers at 128-byte aligned offsets (tensor copies land there);
// 128 bytes of slack align the dynamic base at run time.
constexpr int XY_MAXIN = 4;     // x / y passes: input buffers in the ring at most
constexpr int XY_HEAD = 32;     // ring barriers before the twiddles
__host__ __device__ inline size_t xy_off_in(int twmax, size_t csize) {
    return (XY_HEAD + (size_t)twmax * csize + 127) / 128 * 128;
}
__host__ __device__ inline size_t xy_buf_stride(int bufelems, size_t csize) {
    return ((size_t)bufelems * csize + 127) / 128 * 128;
}
inline size_t xy_smem_bytes(int twmax, int bufelems, int nbuf, size_t csize) {
    return 128 + xy_off_in(twmax, csize) + (size_t)nbuf * xy_buf_stride(bufelems, csize);
}

// stage 1 (x / y): nbuf = buffers in total (ring inputs plus the scratch buffer if any)
size_t stage_smem(int stage, int prec, int n, int tile, int nbuf = 3);
// nab: z-inverse tile buffers (1 when every system of the launch transforms in place)
size_t zinv_smem(int prec, int nzmax, int inelems, int recelems, int abelems, int nab);
size_t contract_smem(int prec, int maxspan);
// Resident blocks per SM a stage's grid is sized for (tile kinds 0..4 as in
// LaunchSet): what the kernel's registers and `smem` bytes of dynamic shared
// memory allow, from the runtime's occupancy calculator (1..8).
int stage_blocks_per_sm(int kind, int prec, size_t smem);
cudaError_t init_kernels(size_t maxsmem);
constexpr int NSTAGE = 9;   // stages per evaluation (stages without tiles are not launched)
constexpr int NKIND = 6;    // tile kinds
// Enqueue all stages; if ev != nullptr, record ev[0..NSTAGE] around them.
cudaError_t launch_all(const LaunchSet &ls, int prec, cudaStream_t st, cudaEvent_t *ev = nullptr);
// one stage: 0 zfwd, 1 plane, 2 yfwd, 3 xfwd, 4 contract, 5 xinv, 6 yinv, 7 zinv, 8 efinish
cudaError_t launch_stage(const LaunchSet &ls, int prec, int stage, cudaStream_t st);
// tile kind a stage walks (-1: efinish, one block per system)
int stage_kind(int stage);
// plane kernel: shared memory per CTA, launch, attributes, clusters per GPU
size_t plane_smem(int nx, int ny, int C);
cudaError_t launch_plane(const LaunchSet &ls, cudaStream_t st);
cudaError_t init_plane_kernel(size_t maxsmem);
int plane_max_clusters(int C, size_t smem);
const char *stage_name(int i);
cudaError_t upload_qmesh(const QMeshDev &q);
// k-point order on the device (plan step): a stable counting sort of the
// half-spectrum k-points of system S (grid, splits and metric set) by
// kernel-table interval into kidx[nx ny (nz/2+1)], with the FP32 interval
// decision of the contraction (f32) or FP64 |k|.  scratch: ksort_scratch_ints
// ints of device memory; its last NK ints receive the k-points per interval.
constexpr int KSORT_RANGE = 16384;   // k-points per warp in the sort
size_t ksort_scratch_ints(size_t nk);
// slab decomposition: x-slab spectrum [xl][P][run] <-> all-to-all send
// buffer [P][xl][run] (run_bytes a multiple of 16)
cudaError_t launch_slab_transpose(const void *src, void *dst, int nxl, int P, size_t run_bytes, bool to_send,
                                  int sms, cudaStream_t st);
cudaError_t launch_ksort(const SysDev &S, bool f32, unsigned *kidx, int *scratch, cudaStream_t st);
cudaError_t launch_q0(int prec, int npts, const double *n, const double *s, double Z, double *q0, double *dqdn,
                      double *dqds);

}  // namespace vdwgb
