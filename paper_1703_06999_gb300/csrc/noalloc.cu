// Evaluation entry point that allocates no memory: for host codes that may
// not call cudaMalloc at the point where they evaluate (for example inside
// their own allocator or memory budget, or in a region where allocation
// calls are forbidden), small grids can be evaluated with all scratch data
// (work buffer, point records, k-point order, energy partials, plan
// descriptors) held in one fixed device array of this file.  The paper's
// method has no counterpart of this; it is a deployment convenience.
//
// The array is a file-scope __device__ array: every GPU that loads this
// library holds it (SCRATCH_BYTES) until the process exits, and every call
// shares it.  Calls that overlap on the GPU (different streams, or a second
// call before the first finished) race on it.  Host code cannot use the
// array's name as a device address: the first call on a device (with that
// device current) asks the runtime for the array's device address once and
// caches it.  The plan data reach the array by copies from pageable host
// memory, so a call may wait for the stream's earlier work before it
// returns, and a call on a stream that is being captured is refused
// (ESTATE): a captured pageable copy would replay from host memory that a
// later call has overwritten.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "table.h"
#include "fftreg.cuh"
#include "contract.cuh"

using namespace vdwgb;

namespace {

constexpr int NA_MAX_AXIS = 64;
constexpr size_t NA_MAX_POINTS = 32768;     // nx * ny * nz
constexpr size_t NA_MAX_KPOINTS = 17408;    // nx * ny * (nz / 2 + 1), e.g. 32 x 32 x 17
constexpr int NA_MAXSPAN = SPAN32;           // kernel-table intervals per contraction chunk
constexpr int NA_CHUNK = CHUNK32;            // k-points per contraction chunk
constexpr int NA_MAX_CHUNKS = (int)(NA_MAX_KPOINTS / NA_CHUNK) + NK / NA_MAXSPAN + 4;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_SPEC = 0;
constexpr size_t OFF_REC = al256(OFF_SPEC + NA_MAX_KPOINTS * NQ * sizeof(cx<float>));
constexpr size_t OFF_KIDX = al256(OFF_REC + NA_MAX_POINTS * sizeof(Rec<float>));
constexpr size_t OFF_CHUNK = al256(OFF_KIDX + NA_MAX_KPOINTS * sizeof(unsigned));
constexpr size_t OFF_EPART = al256(OFF_CHUNK + NA_MAX_CHUNKS * sizeof(int4));
constexpr size_t OFF_TW = al256(OFF_EPART + NA_MAX_CHUNKS * C32_CWARPS * sizeof(double));
constexpr size_t OFF_DESC = al256(OFF_TW + 3 * NA_MAX_AXIS * sizeof(cx<float>));
constexpr size_t OFF_PRE = al256(OFF_DESC + sizeof(SysDev));
constexpr size_t SCRATCH_BYTES = al256(OFF_PRE + 2 * NKIND * sizeof(int));   // about 3.4 MiB

}  // namespace

// the scratch: shared by all calls of vdwgb_calculate_noalloc on a device
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_na_mu;                      // guards the host staging below
unsigned char *g_na_dev[64];             // device address of the scratch, per device
unsigned h_kidx[NA_MAX_KPOINTS];
int h_bin[NA_MAX_KPOINTS];
size_t h_start[NK + 1];
int4 h_chunks[NA_MAX_CHUNKS];
float h_tw[3][2 * NA_MAX_AXIS];

bool radices(int n, AxisPlan &p) {
    int r[32], nr = 0, e2 = 0, m = n;
    while (m % 2 == 0) {
        m /= 2;
        ++e2;
    }
    while (e2 >= 3) { r[nr++] = 8; e2 -= 3; }
    if (e2 == 2) r[nr++] = 4;
    if (e2 == 1) r[nr++] = 2;
    const int odd[3] = {3, 5, 7};
    for (int q : odd)
        while (m % q == 0) {
            r[nr++] = q;
            m /= q;
        }
    if (m != 1 || nr > MAXST) return false;
    p.n = n;
    p.nst = nr;
    for (int i = 0; i < nr; ++i) p.rad[i] = r[i];
    return true;
}

int tile_lines(int stage, int n, int nlines) {
    int best = 1;
    for (int l = 8; l >= 1; --l)
        if (stage_smem(stage, 1, n, l) <= 110 * 1024) { best = l; break; }
    return best > nlines ? nlines : best;
}

int tile_cols(int n, int nzh, int slots) {
    int best = 1;
    for (int w = 8; w >= 1; --w)
        if (stage_smem(1, 1, n, w, slots) <= 110 * 1024) { best = w; break; }
    return best > nzh ? nzh : best;
}

// k-points sorted by kernel-table interval and cut into chunks (same rule as
// the allocating path); returns the chunk count
int sort_chunks(const SysDev &S) {
    const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh;
    const size_t nk = (size_t)nx * ny * nzh;
    for (int j = 0; j <= NK; ++j) h_start[j] = 0;
    auto fold = [](int i, int n) { return i <= (n - 1) / 2 ? i : i - n; };
    for (int px = 0; px < nx; ++px)
        for (int py = 0; py < ny; ++py)
            for (int kz = 0; kz < nzh; ++kz) {
                // frequencies at these positions (the x / y passes may leave them permuted)
                const int x = axis_freq(px, nx, S.sx1), y = axis_freq(py, ny, S.sy1);
                const int mx = fold(x, nx), my = fold(y, ny);
                const bool qx = (nx % 2 == 0) && (x == nx / 2), qy = (ny % 2 == 0) && (y == ny / 2);
                const bool qz = (nz % 2 == 0) && (kz == nz / 2);
                const int mz = qz ? -kz : kz;
                int j;                           // the FP32 decision the contraction repeats
                float tt;
                kpoint_interval32(S.gf, mx, my, mz, qx, qy, qz, j, tt);
                const size_t idx = ((size_t)px * ny + py) * nzh + kz;
                h_bin[idx] = (int)j;
                ++h_start[j + 1];
            }
    for (int j = 1; j <= NK; ++j) h_start[j] += h_start[j - 1];
    for (size_t i = 0; i < nk; ++i) h_kidx[h_start[h_bin[i]]++] = (unsigned)i;   // h_start[j] -> end of bin j
    int nch = 0;
    size_t i = 0;
    while (i < nk && nch < NA_MAX_CHUNKS) {
        const int j0 = h_bin[h_kidx[i]];
        size_t n = 0;
        int jl = j0;
        while (i + n < nk && n < (size_t)NA_CHUNK) {
            const int jb = h_bin[h_kidx[i + n]];
            if (j0 == NK - 1 ? jb != NK - 1 : (jb == NK - 1 || jb - j0 >= NA_MAXSPAN)) break;
            jl = jb;
            ++n;
        }
        h_chunks[nch++] = make_int4((int)i, (int)n, j0, j0 == NK - 1 ? 0 : jl - j0 + 1);
        i += n;
    }
    return i < nk ? -1 : nch;
}

}  // namespace

extern "C" int vdwgb_calculate_noalloc(int device, int functional, int nx, int ny, int nz, const double *cell9,
                                       const double *d_rho, const double *d_sigma, double *d_dedrho,
                                       double *d_dedsigma, double *d_energy, void *cuda_stream) {
    if (!cell9 || !d_rho || !d_sigma || !d_dedrho || !d_dedsigma || !d_energy)
        return fail(VDWGB_EINVAL, "null argument");
    if (functional != VDWGB_DF1 && functional != VDWGB_DF2) return fail(VDWGB_EINVAL, "unknown functional");
    if (nx < 1 || ny < 1 || nz < 1 || nx > NA_MAX_AXIS || ny > NA_MAX_AXIS || nz > NA_MAX_AXIS ||
        (size_t)nx * ny * nz > NA_MAX_POINTS || (size_t)nx * ny * (nz / 2 + 1) > NA_MAX_KPOINTS)
        return fail(VDWGB_EINVAL,
                    "grid %dx%dx%d beyond the fixed scratch: axes <= %d, nx*ny*nz <= %zu, nx*ny*(nz/2+1) <= %zu",
                    nx, ny, nz, NA_MAX_AXIS, NA_MAX_POINTS, NA_MAX_KPOINTS);
    int sms = 0;
    size_t maxsmem = 0;
    int *err = nullptr;
    TableRefs tr;
    if (!device_peek(device, &sms, &maxsmem, &err) || !table_peek(device, tr))
        return fail(VDWGB_ESTATE,
                    "device %d has no resident kernel table yet: build it once with vdwgb_kernel_table "
                    "(which allocates) before calling vdwgb_calculate_noalloc", device);
    SysDev S;
    std::memset(&S, 0, sizeof S);
    S.nx = nx;
    S.ny = ny;
    S.nz = nz;
    S.nzh = nz / 2 + 1;
    S.nyg = ny;
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        if (!radices(dims[a], S.ax[a]))
            return fail(VDWGB_EINVAL, "axis %d length %d: prime factors must be 2, 3, 5, 7", a, dims[a]);
    const double *c = cell9;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    if (!(std::fabs(det) > 1e-12)) return fail(VDWGB_EINVAL, "cell volume is zero");
    double inv[9];
    inv[0] = (c[4] * c[8] - c[5] * c[7]) / det;
    inv[1] = (c[2] * c[7] - c[1] * c[8]) / det;
    inv[2] = (c[1] * c[5] - c[2] * c[4]) / det;
    inv[3] = (c[5] * c[6] - c[3] * c[8]) / det;
    inv[4] = (c[0] * c[8] - c[2] * c[6]) / det;
    inv[5] = (c[2] * c[3] - c[0] * c[5]) / det;
    inv[6] = (c[3] * c[7] - c[4] * c[6]) / det;
    inv[7] = (c[1] * c[6] - c[0] * c[7]) / det;
    inv[8] = (c[0] * c[4] - c[1] * c[3]) / det;
    double B[9];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) B[j * 3 + k] = 2.0 * M_PI * inv[k * 3 + j];
    auto gdot = [&](int i, int j) { return B[i * 3] * B[j * 3] + B[i * 3 + 1] * B[j * 3 + 1] + B[i * 3 + 2] * B[j * 3 + 2]; };
    S.g[0] = gdot(0, 0);
    S.g[1] = gdot(1, 1);
    S.g[2] = gdot(2, 2);
    S.g[3] = gdot(0, 1);
    S.g[4] = gdot(0, 2);
    S.g[5] = gdot(1, 2);
    for (int i = 0; i < 6; ++i) S.gf[i] = (float)S.g[i];
    const double N = (double)nx * ny * nz;
    S.escale = 0.5 * std::fabs(det) / (N * N);
    S.invN = 1.0 / N;
    S.Z = functional == VDWGB_DF2 ? -1.887 : -0.8491;
    {
        const double zc = -S.Z / 36.0;
        S.zc[0] = (float)zc;
        S.zc[1] = (float)(zc - (double)S.zc[0]);
    }
    S.invNf = (float)S.invN;
    // tiles: the same rules as the allocating path without autotuning
    const int nzh = S.nzh;
    S.LZ = tile_lines(0, nz, nx * ny);
    S.LZi = tile_lines(3, nz, nx * ny);
    S.sx1 = xy_split(nx);                    // in-place x / y transforms where compiled
    S.sy1 = xy_split(ny);
    S.sz1 = fft_split(nz);
    const int workx = S.sx1 ? 0 : 1, worky = S.sy1 ? 0 : 1;
    S.Wy = tile_cols(ny, nzh, 2 + worky);
    S.Wx = tile_cols(nx, nzh, 2 + workx);
    S.tiles[0] = (nx * ny + S.LZ - 1) / S.LZ;
    S.tiles[1] = nx * ((nzh + S.Wy - 1) / S.Wy);
    S.tiles[2] = ny * ((nzh + S.Wx - 1) / S.Wx);
    S.tiles[3] = (nx * ny + S.LZi - 1) / S.LZi;

    std::lock_guard<std::mutex> lk(g_na_mu);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(VDWGB_ESTATE, "vdwgb_calculate_noalloc cannot run on a stream that is being captured");
    }
    if (!g_na_dev[device]) {
        // once per device, with the device current: the array's device address
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
        g_na_dev[device] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *base = g_na_dev[device];
    const int nch = sort_chunks(S);
    if (nch < 0) return fail(VDWGB_EINVAL, "too many contraction chunks for the fixed scratch");
    S.tiles[4] = nch;
    S.nepart = nch * C32_CWARPS;             // one energy partial per chunk and consumer warp
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < dims[a]; ++m) {
            const double ang = 2.0 * M_PI * (double)m / (double)dims[a];
            h_tw[a][2 * m] = (float)std::cos(ang);
            h_tw[a][2 * m + 1] = (float)-std::sin(ang);
        }
    S.spec = base + OFF_SPEC;
    S.rec = base + OFF_REC;
    S.kidx = reinterpret_cast<const unsigned *>(base + OFF_KIDX);
    S.chunks = reinterpret_cast<const int4 *>(base + OFF_CHUNK);
    S.epart = reinterpret_cast<double *>(base + OFF_EPART);
    for (int a = 0; a < 3; ++a) S.tw[a] = base + OFF_TW + (size_t)a * NA_MAX_AXIS * sizeof(cx<float>);
    S.err = err;
    S.n = d_rho;
    S.sigma = d_sigma;
    S.dedn = d_dedrho;
    S.dedsigma = d_dedsigma;
    S.energy = d_energy;
    int pre[2 * NKIND];
    for (int k = 0; k < NKIND; ++k) {
        pre[2 * k] = 0;
        pre[2 * k + 1] = S.tiles[k];
    }
    // launch set (FP32-mixed, cubic interpolation)
    LaunchSet L;
    std::memset(&L, 0, sizeof L);
    L.sys = reinterpret_cast<const SysDev *>(base + OFF_DESC);
    L.nsys = 1;
    L.maxspan = NA_MAXSPAN;
    L.err = err;
    L.table = tr.cub32;
    const int *dpre = reinterpret_cast<const int *>(base + OFF_PRE);
    for (int k = 0; k < NKIND; ++k) {
        L.prefix[k] = dpre + 2 * k;
        L.total[k] = S.tiles[k];
    }
    L.twmax[0] = L.twmax[3] = nz;
    L.twmax[1] = ny;
    L.twmax[2] = nx;
    L.bufelems[3] = 0;                               // FP32: direct z-inverse, nothing staged
    L.recelems = 0;
    L.abelems = nz * z_ld(S.LZi);
    L.bufelems[1] = ny * S.Wy * NQ;
    L.bufelems[2] = nx * S.Wx * NQ;
    L.nbuf[1] = L.nbuf[2] = 2;
    L.work[0] = S.sz1 ? 0 : 1;
    L.work[1] = worky;
    L.work[2] = workx;
    L.work[3] = L.work[0];
    L.smem[0] = stage_smem(0, 1, nz, S.LZ);
    L.smem[1] = stage_smem(1, 1, ny, S.Wy, 2 + worky);
    L.smem[2] = stage_smem(1, 1, nx, S.Wx, 2 + workx);
    L.smem[3] = stage_smem(3, 1, nz, S.LZi);
    L.smem[4] = contract_smem(1, NA_MAXSPAN);
    for (int k = 0; k < NKIND; ++k) {
        if (L.smem[k] > maxsmem - 1024) return fail(VDWGB_EINVAL, "tile does not fit shared memory");
        const int cap = sms * stage_blocks_per_sm(k, 1, L.smem[k]);
        L.grid[k] = L.total[k] < cap ? L.total[k] : cap;
    }
    // uploads from host staging (pageable: each copy has read its source when it returns)
    const size_t nk = (size_t)nx * ny * nzh;
    e = cudaMemcpyAsync(base + OFF_KIDX, h_kidx, nk * sizeof(unsigned), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + OFF_CHUNK, h_chunks, nch * sizeof(int4), cudaMemcpyHostToDevice, st);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(base + OFF_TW + (size_t)a * NA_MAX_AXIS * sizeof(cx<float>), h_tw[a],
                            dims[a] * sizeof(cx<float>), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + OFF_DESC, &S, sizeof S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + OFF_PRE, pre, sizeof pre, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_all(L, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc evaluation");
    return 0;
}
