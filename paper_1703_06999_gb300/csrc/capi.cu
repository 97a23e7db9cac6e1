// C ABI of the library (include/vdwgb.h): handles, FFT plans, launches,
// batches.  Host code only; the kernels are in pipeline.cu and table.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>
#include <map>
#include <tuple>
#include <cstdlib>
#include <algorithm>
#include <atomic>

#include <cuda.h>

#include "internal.h"
#include "table.h"
#include "fftreg.cuh"
#include "contract.cuh"

using namespace vdwgb;

static thread_local std::string g_err;

namespace vdwgb {
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(VDWGB_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(VDWGB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace vdwgb

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------
// per-device one-time setup: q-mesh constants, kernel shared-memory limits
// ---------------------------------------------------------------------------
struct DevInfo {
    bool ready = false;
    int sms = 0;
    size_t maxsmem = 0;
    size_t smem_sm = 0;      // shared memory per SM
    int *err = nullptr;      // device flag written by kernels whose bounded wait ran out
};
static std::mutex g_dev_mu;
static DevInfo g_dev[64];

int vdwgb::device_setup(int device) {
    if (device < 0 || device >= 64) return fail(VDWGB_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevInfo &d = g_dev[device];
    if (d.ready) return 0;
    CK(cudaSetDevice(device), "cudaSetDevice");
    int sms = 0, optin = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "attr");
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device), "attr");
    int smsm = 0;
    CK(cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device), "attr");
    d.sms = sms;
    d.maxsmem = (size_t)optin;
    d.smem_sm = (size_t)smsm;
    QMeshDev qm;
    host_qmesh(qm);
    CK(upload_qmesh(qm), "upload q-mesh");
    CK(init_kernels(d.maxsmem - 1024), "kernel attributes");
    CK(cudaMalloc(&d.err, 2 * sizeof(int)), "error flag");     // status, detail
    CK(cudaMemset(d.err, 0, 2 * sizeof(int)), "error flag");
    d.ready = true;
    return 0;
}

// Set-up state of a device if vdwgb_* set it up earlier (never sets up or
// allocates).
bool vdwgb::device_peek(int device, int *sms, size_t *maxsmem, int **err) {
    if (device < 0 || device >= 64) return false;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    const DevInfo &d = g_dev[device];
    if (!d.ready) return false;
    *sms = d.sms;
    *maxsmem = d.maxsmem;
    *err = d.err;
    return true;
}

// ---------------------------------------------------------------------------
// FFT plan of one axis
// ---------------------------------------------------------------------------
static bool factor_axis(int n, AxisPlan &p) {
    p.n = n;
    p.nst = 0;
    int e2 = 0, m = n;
    while (m % 2 == 0) { m /= 2; ++e2; }
    std::vector<int> r;
    while (e2 >= 3) { r.push_back(8); e2 -= 3; }
    if (e2 == 2) r.push_back(4);
    if (e2 == 1) r.push_back(2);
    const int odd[3] = {3, 5, 7};
    for (int q : odd)
        while (m % q == 0) { r.push_back(q); m /= q; }
    if (m != 1 || (int)r.size() > MAXST) return false;
    p.nst = (int)r.size();
    for (int i = 0; i < p.nst; ++i) p.rad[i] = r[i];
    return true;
}

static std::vector<double> twiddles(int n) {
    std::vector<double> w(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        // exp(-2 pi i m / n), argument reduced to the first half-turn for accuracy
        const double ang = 2.0 * M_PI * (double)m / (double)n;
        w[2 * m] = std::cos(ang);
        w[2 * m + 1] = -std::sin(ang);
    }
    return w;
}

// ---------------------------------------------------------------------------
// handle (struct vdwgb_data in internal.h)
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Fault injection (vdwgb_inject_fault): armed counts, taken one at a time
// ---------------------------------------------------------------------------
static std::atomic<int> g_inj_alloc{0}, g_inj_wait{0};

static bool take_injection(std::atomic<int> &c) {
    int v = c.load();
    while (v > 0)
        if (c.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

// cudaMalloc, or the out-of-memory error an armed injection asks for
cudaError_t vdwgb::device_malloc(void **p, size_t bytes) {
    if (take_injection(g_inj_alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

static cudaError_t dalloc(vdwgb_data *h, void **p, size_t bytes) {
    if (take_injection(g_inj_alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (h->alloc_stream) return cudaMallocAsync(p, bytes, h->alloc_stream);
    return cudaMalloc(p, bytes);
}
template <typename P>
static cudaError_t dalloc(vdwgb_data *h, P **p, size_t bytes) {
    return dalloc(h, reinterpret_cast<void **>(p), bytes);
}
static cudaError_t dupload(vdwgb_data *h, void *dst, const void *src, size_t bytes) {
    if (h->alloc_stream) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->alloc_stream);
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}
static void dfree(vdwgb_data *h, void *p) {
    if (!p) return;
    if (h->alloc_stream) cudaFreeAsync(p, h->alloc_stream);
    else cudaFree(p);
}

static void release(vdwgb_data *h) {
    if (!h) return;
    if (h->device >= 0) cudaSetDevice(h->device);
    if (!h->spec_external) dfree(h, h->spec);
    h->spec_external = false;
    dfree(h, h->rec);
    dfree(h, h->epart);
    for (int i = 0; i < 3; ++i) dfree(h, h->tw[i]);
    dfree(h, h->kidx);
    dfree(h, h->chunks);
    dfree(h, h->kord);
    dfree(h, h->tmap);
    h->tmap = nullptr;
    h->kidx = nullptr;
    h->chunks = nullptr;
    h->kord = nullptr;
    dfree(h, h->dsys);
    dfree(h, h->dprefix);
    dfree(h, h->d_io);
    table_custom_free(h->ktab);
    dfree(h, h->d_spin);
    dfree(h, h->d_spin_io);
    h->d_spin = h->d_spin_io = nullptr;
    if (h->stream) cudaStreamDestroy(h->stream);
    h->spec = h->rec = nullptr;
    h->epart = nullptr;
    h->dsys = nullptr;
    h->dprefix = nullptr;
    h->d_io = nullptr;
    h->stream = nullptr;
    for (int i = 0; i < 3; ++i) h->tw[i] = nullptr;
    h->inited = false;
}

static size_t elem_bytes(int prec) { return prec == VDWGB_FP32_MIXED ? 8 : 16; }
static size_t rec_bytes(int prec) { return prec == VDWGB_FP32_MIXED ? 16 : 32; }

// Default tile choices (heuristic): z passes LZ / LZi lines, y / x passes Wy /
// Wx kz-columns with three row buffers (prefetch); prefer two blocks per SM
// (<= ~110 KB).  Axes too long for three buffers of one column use two (no
// prefetch).  The autotuner below replaces them by measured choices.
static const size_t TILE_BUDGET = 110 * 1024;

// Caps on one tile's shared memory, default and autotuned tiles alike.  A
// batch launch takes the largest tile of its systems, so one system's large
// tile would set every system's occupancy: FP32 x / y tiles are kept to two
// blocks per SM and z tiles to three (the blocks the kernels' register
// bounds allow), each block with its static shared memory and the 1 KB the
// runtime reserves.  FP64 kernels run one block per SM: no cap.
// VDWGB_XY_CAP / VDWGB_Z_CAP (bytes) override.  Measured on the 64 uneven
// grids: x / y passes 1.31 -> 0.94 ms, z inverse 1.44 -> 1.28 ms.
static void tile_caps(int device, int prec, size_t &xy, size_t &z) {
    static size_t env[2] = {0, 0};
    static std::once_flag once;
    std::call_once(once, [] {
        const char *e[2] = {std::getenv("VDWGB_XY_CAP"), std::getenv("VDWGB_Z_CAP")};
        for (int i = 0; i < 2; ++i) env[i] = e[i] ? (size_t)std::strtoull(e[i], nullptr, 10) : 0;
    });
    const size_t sm = g_dev[device].smem_sm;
    const bool f32 = prec == VDWGB_FP32_MIXED && sm > 0;
    xy = env[0] ? env[0] : (f32 ? sm / 2 - 2560 : (size_t)-1);
    z = env[1] ? env[1] : (f32 ? sm / 3 - 1824 : (size_t)-1);
}

// The z cap for one z stage (0 forward, 3 inverse) of an axis of nz points:
// where it would leave tiles of a single line (long axes: 640 points take
// about 100 KB per two lines), tiles of one line cost more than the lost
// occupancy, and the stage keeps the uncapped limit.
static size_t z_stage_cap(int stage, int prec, int nz, size_t zcap, size_t lim) {
    return stage_smem(stage, prec, nz, 2) <= zcap ? std::min(zcap, lim) : lim;
}


static int best_w(int prec, int n, int nzh, int slots, size_t budget) {
    int W = 1;
    for (int w = 8; w >= 1; --w)
        if (stage_smem(1, prec, n, w, slots) <= budget) { W = w; break; }
    return W > nzh ? nzh : W;
}

// x / y passes: two ring buffers (one tile prefetched) plus the scratch
// buffer on axes without an in-place transform (workx / worky)
static void choose_tiles(int prec, int nx, int ny, int nz, int nzh, size_t lim, size_t xycap, size_t zcap,
                         int workx, int worky, int &LZ, int &LZi, int &Wy, int &Wx, int &nbuf) {
    const size_t xybudget = std::min(TILE_BUDGET, xycap);
    const size_t zb0 = std::min(TILE_BUDGET, z_stage_cap(0, prec, nz, zcap, lim));
    const size_t zb3 = std::min(TILE_BUDGET, z_stage_cap(3, prec, nz, zcap, lim));
    LZ = 1;
    for (int l = 16; l >= 1; --l)
        if (stage_smem(0, prec, nz, l) <= zb0) { LZ = l; break; }
    LZi = 1;
    for (int l = 16; l >= 1; --l)
        if (stage_smem(3, prec, nz, l) <= zb3) { LZi = l; break; }
    if (LZi > nx * ny) LZi = nx * ny;
    if (LZ > nx * ny) LZ = nx * ny;
    nbuf = 2;
    if (stage_smem(1, prec, ny, 1, 2 + worky) > lim || stage_smem(1, prec, nx, 1, 2 + workx) > lim) nbuf = 1;
    Wy = best_w(prec, ny, nzh, nbuf + worky, xybudget);
    Wx = best_w(prec, nx, nzh, nbuf + workx, xybudget);
}

// Contraction chunks of a system from the k-points per kernel-table interval
// of its sorted order (the order is interval by interval, so the counts fix
// it): chunks of at most `chunkmax` k-points spanning at most `maxspan`
// intervals; k-points beyond the table (interval NK - 1) form their own
// chunks.  chunk = {first index into the order, count, first interval,
// intervals staged (0 beyond the table)}.
static void chunks_from_counts(const std::vector<int> &count, int maxspan, int chunkmax, std::vector<int4> &chunks) {
    chunks.clear();
    int j = 0;
    while (j < NK && count[j] == 0) ++j;
    int left = j < NK ? count[j] : 0;   // k-points of interval j not yet in a chunk
    size_t pos = 0;
    while (j < NK) {
        const int j0 = j;
        int n = 0, jl = j0;
        while (j < NK && n < chunkmax) {
            if (j0 == NK - 1 ? j != NK - 1 : (j == NK - 1 || j - j0 >= maxspan)) break;
            const int take = std::min(left, chunkmax - n);
            n += take;
            left -= take;
            jl = j;
            if (left == 0) {
                ++j;
                while (j < NK && count[j] == 0) ++j;
                left = j < NK ? count[j] : 0;
            }
        }
        chunks.push_back(make_int4((int)pos, n, j0, j0 == NK - 1 ? 0 : jl - j0 + 1));
        pos += (size_t)n;
    }
}

// Upper bound of the chunk count of any system of nk k-points.
static size_t max_chunks(size_t nk, int chunkmax) { return (nk + chunkmax - 1) / chunkmax + NK + 1; }

// Reciprocal metric, energy scale and functional constants of the handle's
// cell and functional in its descriptor.
static void set_metric(vdwgb_data *h) {
    SysDev &S = h->hsys;
    const double *c = h->cell;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    double inv[9];   // inverse of C
    inv[0] = (c[4] * c[8] - c[5] * c[7]) / det;
    inv[1] = (c[2] * c[7] - c[1] * c[8]) / det;
    inv[2] = (c[1] * c[5] - c[2] * c[4]) / det;
    inv[3] = (c[5] * c[6] - c[3] * c[8]) / det;
    inv[4] = (c[0] * c[8] - c[2] * c[6]) / det;
    inv[5] = (c[2] * c[3] - c[0] * c[5]) / det;
    inv[6] = (c[3] * c[7] - c[4] * c[6]) / det;
    inv[7] = (c[1] * c[6] - c[0] * c[7]) / det;
    inv[8] = (c[0] * c[4] - c[1] * c[3]) / det;
    double B[9];   // reciprocal lattice, B = 2 pi C^{-T} (rows b_j): B[j][k] = 2 pi inv[k][j]
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) B[j * 3 + k] = 2.0 * M_PI * inv[k * 3 + j];
    double g[3][3];  // g = B B^T: |k|^2 = m^T g m
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            g[i][j] = B[i * 3] * B[j * 3] + B[i * 3 + 1] * B[j * 3 + 1] + B[i * 3 + 2] * B[j * 3 + 2];
    S.g[0] = g[0][0];
    S.g[1] = g[1][1];
    S.g[2] = g[2][2];
    S.g[3] = g[0][1];
    S.g[4] = g[0][2];
    S.g[5] = g[1][2];
    for (int i = 0; i < 6; ++i) S.gf[i] = (float)S.g[i];
    const double N = (double)S.nx * S.ny * S.nz;
    S.escale = 0.5 * std::fabs(det) / (N * N);
    S.invN = 1.0 / N;
    S.Z = h->functional == VDWGB_DF2 ? -1.887 : -0.8491;
    const double zc = -S.Z / 36.0;
    S.zc[0] = (float)zc;
    S.zc[1] = (float)(zc - (double)S.zc[0]);
    S.invNf = (float)S.invN;
}

// The k-point order of the handle's current cell, sorted on the device into
// h->kidx (stream st, spec buffer as scratch when large enough), and its
// chunks uploaded to h->chunks (capacity max_chunks).  Sets tiles[4] and
// nepart.  Waits for st (the interval counts come back to the host).
static int sort_kpoints(vdwgb_data *h, cudaStream_t st) {
    SysDev &S = h->hsys;
    const bool f32 = h->prec == VDWGB_FP32_MIXED;
    const int maxspan = f32 ? SPAN32 : SPAN64;
    const int chunkmax = f32 ? CHUNK32 : CHUNK64;
    const size_t nk = (size_t)S.nx * S.ny * S.nzh;
    const size_t need = ksort_scratch_ints(nk) * sizeof(int);
    const size_t specbytes = nk * NQ * elem_bytes(h->prec);
    int *scratch = nullptr;
    if (need <= specbytes) scratch = static_cast<int *>(h->spec);
    else CK(dalloc(h, &scratch, need), "k-point sort scratch");
    std::vector<int> count(NK, 0);
    cudaError_t e = launch_ksort(S, f32, h->kidx, scratch, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(count.data(), scratch + (need / sizeof(int) - NK), NK * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (scratch != h->spec) dfree(h, scratch);
    if (e != cudaSuccess) return cuda_fail(e, "k-point sort");
    std::vector<int4> chunks;
    chunks_from_counts(count, maxspan, chunkmax, chunks);
    if (chunks.size() > max_chunks(nk, chunkmax)) return fail(VDWGB_ECUDA, "k-point sort: chunk bound exceeded");
    CK(cudaMemcpyAsync(h->chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, st), "chunks");
    CK(cudaStreamSynchronize(st), "chunks");   // the host vector is released on return
    S.tiles[4] = (int)chunks.size();
    S.nepart = S.tiles[4] * (f32 ? C32_CWARPS : 1);   // FP32: one per consumer warp
    LaunchSet &L = h->ls;
    L.total[4] = S.tiles[4];
    const int cap = g_dev[h->device].sms * stage_blocks_per_sm(4, h->prec, L.smem[4]);
    L.grid[4] = L.total[4] < cap ? L.total[4] : cap;
    return 0;
}

// ---------------------------------------------------------------------------
// Fused plane kernel: eligibility and the per-(kz, rank) k-point order
// ---------------------------------------------------------------------------
static int g_fused = -1;   // -1: read VDWGB_FUSED once (default off)
static std::mutex g_fused_mu;

static bool fused_on() {
    std::lock_guard<std::mutex> lk(g_fused_mu);
    if (g_fused < 0) {
        const char *e = std::getenv("VDWGB_FUSED");
        g_fused = (e && e[0] == '1') ? 1 : 0;
    }
    return g_fused == 1;
}

// Cluster size for the plane kernel on this system (16), 0 if it takes the
// separate y / x / contraction passes: FP32-mixed, both in-plane axes with a
// two-pass split and divisible by C, one chunk small enough for the swap
// registers (XL YL 20 <= 3072), nx YL < 65536, the CTA's share of the plane in shared memory.
static int fused_cluster(const vdwgb_data *h, size_t lim, int &maxcl) {
    maxcl = 0;
    if (h->prec != VDWGB_FP32_MIXED || !fused_on()) return 0;
    const int nx = h->nx, ny = h->ny;
    if (!fft_split(nx) || !fft_split(ny)) return 0;
    const int cand[1] = {16};         // one cluster size, so any fused systems share a launch
    for (int C : cand) {
        if (nx % C || ny % C) continue;
        const int XL = nx / C, YL = ny / C;
        if (XL * YL * NQ > 3072 || nx * YL > 65535) continue;     // swap registers; 16-bit k-point ids
        const size_t sm = plane_smem(nx, ny, C);
        if (sm > lim - 64) continue;
        const int m = plane_max_clusters(C, sm);
        if (m < 1) continue;
        maxcl = m;
        return C;
    }
    return 0;
}

// kord: for each kz and rank, the local indices px YL + yl of the rank's
// k-points (x position px, y position rank YL + yl, both in the permuted
// order of the in-place transforms), sorted by kernel-table interval
static void build_kord(const SysDev &S, int C, std::vector<unsigned short> &kord, int &kstride) {
    const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh;
    const int YL = ny / C;
    const int n1x = fft_split(nx), n2x = nx / n1x, n1y = fft_split(ny), n2y = ny / n1y;
    const int npts = nx * YL;
    kstride = (npts + 7) & ~7;
    kord.assign((size_t)nzh * C * kstride, 0);
    const double dk = 2.0 * M_PI / RMAX;
    std::vector<int> bin(npts);
    std::vector<int> start(NK + 1);
    auto fold = [](int i, int n) { return i <= (n - 1) / 2 ? i : i - n; };
    for (int kz = 0; kz < nzh; ++kz) {
        const bool qz = (nz % 2 == 0) && (kz == nz / 2);
        const int mz = qz ? -kz : kz;
        const double cz = qz ? 0.0 : mz;
        for (int c = 0; c < C; ++c) {
            std::fill(start.begin(), start.end(), 0);
            for (int li = 0; li < npts; ++li) {
                const int px = li / YL, yl = li % YL;
                const int x = fft_perm_freq(px, n1x, n2x), y = fft_perm_freq(c * YL + yl, n1y, n2y);
                const int mx = fold(x, nx), my = fold(y, ny);
                const bool qx = (nx % 2 == 0) && (x == nx / 2), qy = (ny % 2 == 0) && (y == ny / 2);
                const double cx = qx ? 0.0 : mx, cy = qy ? 0.0 : my;
                double k2 = S.g[0] * mx * mx + S.g[1] * (double)my * my + S.g[2] * (double)mz * mz +
                            2.0 * (S.g[3] * cx * cy + S.g[4] * cx * cz + S.g[5] * cy * cz);
                if (k2 < 0) k2 = 0;
                long j = (long)(std::sqrt(k2) / dk);
                if (j > NK - 1) j = NK - 1;
                bin[li] = (int)j;
                ++start[j + 1];
            }
            for (int j = 1; j <= NK; ++j) start[j] += start[j - 1];
            unsigned short *out = kord.data() + ((size_t)kz * C + c) * kstride;
            for (int li = 0; li < npts; ++li) out[start[bin[li]]++] = (unsigned short)li;
        }
    }
}

// kernel launches one evaluation of a launch set enqueues (stages without tiles are skipped)
static int count_launches(const LaunchSet &L) {
    int n = 0;
    for (int k = 0; k < NSTAGE; ++k) {
        const int kind = stage_kind(k);
        if (kind < 0 || L.total[kind] > 0) ++n;
    }
    return n;
}

// Tile-dependent parts of a handle's plan: tile counts of the z, y, x passes
// and the matching launch-set fields.
static void set_tiles(vdwgb_data *h, int LZ, int LZi, int Wy, int Wx, int nby, int nbx) {
    SysDev &S = h->hsys;
    LaunchSet &L = h->ls;
    const int prec = h->prec;
    const int nx = S.nx, ny = S.ny, nz = S.nz, nzh = S.nzh;
    DevInfo &di = g_dev[h->device];
    S.LZ = LZ;
    S.LZi = LZi;
    S.Wy = Wy;
    S.Wx = Wx;
    S.tiles[0] = (nx * ny + LZ - 1) / LZ;
    S.tiles[1] = S.fused ? 0 : nx * ((nzh + Wy - 1) / Wy);
    S.tiles[2] = S.fused ? 0 : ny * ((nzh + Wx - 1) / Wx);
    S.tiles[3] = (nx * ny + LZi - 1) / LZi;
    for (int s = 0; s < 4; ++s) {
        L.prefix[s] = h->dprefix + 2 * s;
        L.total[s] = S.tiles[s];
    }
    L.twmax[0] = L.twmax[3] = nz;
    L.twmax[1] = ny;
    L.twmax[2] = nx;
    L.bufelems[0] = 0;
    // z-inverse: FP32 reads the spectrum and the records straight from
    // global memory (nothing staged); FP64 stages tiles
    const bool zdirect = prec == VDWGB_FP32_MIXED;
    L.bufelems[3] = zdirect ? 0 : LZi * nzh * NQ;
    L.recelems = zdirect ? 0 : LZi * nz;
    L.abelems = nz * z_ld(LZi);
    L.bufelems[1] = ny * Wy * NQ;
    L.bufelems[2] = nx * Wx * NQ;
    L.nbuf[0] = L.nbuf[3] = 0;
    L.nbuf[1] = nby;
    L.nbuf[2] = nbx;
    L.work[0] = S.sz1 ? 0 : 1;
    L.work[1] = S.sy1 ? 0 : 1;
    L.work[2] = S.sx1 ? 0 : 1;
    L.work[3] = L.work[0];
    L.smem[0] = stage_smem(0, prec, nz, LZ);
    L.smem[3] = stage_smem(3, prec, nz, LZi);
    L.smem[1] = stage_smem(1, prec, ny, Wy, nby + L.work[1]);
    L.smem[2] = stage_smem(1, prec, nx, Wx, nbx + L.work[2]);
    for (int s = 0; s < 4; ++s) {
        const int cap = di.sms * stage_blocks_per_sm(s, prec, L.smem[s]);
        L.grid[s] = L.total[s] < cap ? L.total[s] : cap;
    }
}

// ---------------------------------------------------------------------------
// Tensor maps of the spectrum for the x / y passes (FP32): a 3-D view
// [x][y][kz 20 + a] of 8-byte complex values; the y-pass box is W_y 20 x ny x 1
// at (kz0 20, 0, x), the x-pass box W_x 20 x 1 x nx at (kz0 20, y, 0).  The
// encoder comes from the driver through the runtime (no link to libcuda).
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Rows per tensor copy of a tile of n rows and W kz-columns: n itself up to
// 256 (one copy), else the largest divisor of n <= 256 whose copies land at
// 128-byte aligned offsets of the tile buffer (rows x W x 20 x 8 bytes), at
// most 16 copies; 0: none (row-by-row copies).
static int tile_box_rows(int n, int W) {
    if (n <= 256) return n;
    for (int k = 2; k <= 16; ++k) {
        if (n % k) continue;
        const int b = n / k;
        if (b <= 256 && (b * W) % 4 == 0) return b;
    }
    return 0;
}

// both maps of a handle's current plan; false if a box does not fit the
// tensor-copy limits (each box side <= 256) or no encoder is available.
// by / bx: rows per copy of a y / x tile
static bool encode_xy_maps(const SysDev &S, CUtensorMap maps[2], int &by, int &bx) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !S.spec) return false;
    const int nzh = S.nzh;
    if (S.Wy * NQ > 256 || S.Wx * NQ > 256) return false;
    by = tile_box_rows(S.ny, S.Wy);
    bx = tile_box_rows(S.nx, S.Wx);
    if (!by || !bx) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nzh * NQ, (cuuint64_t)S.ny, (cuuint64_t)S.nx};
    const cuuint64_t strides[2] = {(cuuint64_t)nzh * NQ * 8, (cuuint64_t)S.ny * nzh * NQ * 8};
    const cuuint32_t one[3] = {1, 1, 1};
    const cuuint32_t box_y[3] = {(cuuint32_t)(S.Wy * NQ), (cuuint32_t)by, 1};
    const cuuint32_t box_x[3] = {(cuuint32_t)(S.Wx * NQ), 1, (cuuint32_t)bx};
    for (int m = 0; m < 2; ++m) {
        const CUresult r = enc(&maps[m], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, S.spec, dims, strides,
                               m == 0 ? box_y : box_x, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

// encode the maps for the current tiles and point the descriptor at them (or
// clear the pointer: row-by-row copies)
static int upload_maps(vdwgb_data *h, bool sync) {
    SysDev &S = h->hsys;
    S.tmap = nullptr;
    S.tby = S.tbx = 0;
    if (!h->tmap) return 0;
    alignas(64) CUtensorMap maps[2];
    int by = 0, bx = 0;
    if (!encode_xy_maps(S, maps, by, bx)) return 0;
    if (sync) CK(cudaMemcpy(h->tmap, maps, sizeof maps, cudaMemcpyHostToDevice), "tensor maps");
    else CK(dupload(h, h->tmap, maps, sizeof maps), "tensor maps");
    S.tmap = h->tmap;
    S.tby = by;
    S.tbx = bx;
    return 0;
}

static int upload_plan(vdwgb_data *h) {
    {
        const int rc = upload_maps(h, false);
        if (rc) return rc;
    }
    int pre[2 * NKIND];
    for (int s = 0; s < NKIND; ++s) {
        pre[2 * s] = 0;
        pre[2 * s + 1] = h->hsys.tiles[s];
    }
    CK(dupload(h, h->dprefix, pre, sizeof pre), "prefix");
    CK(dupload(h, h->dsys, &h->hsys, sizeof(SysDev)), "descriptor");
    h->last_ptr[0] = nullptr;   // descriptor rewritten: refresh I/O pointers next call
    return 0;
}

// ---------------------------------------------------------------------------
// Autotuner: per (grid, precision) the tile shapes LZ (z forward), Wy, Wx
// (y, x passes) and LZi (z inverse) are chosen by timing each stage on the
// device for every candidate that fits shared memory; results are cached for
// the process.  Enabled by vdwgb_set_autotune(1) or VDWGB_AUTOTUNE=1.
// ---------------------------------------------------------------------------
struct TuneKey {
    int nx, ny, nz, prec;
    bool operator<(const TuneKey &o) const {
        return std::tie(nx, ny, nz, prec) < std::tie(o.nx, o.ny, o.nz, o.prec);
    }
};
struct TuneVal {
    int LZ, LZi, Wy, Wx, nby, nbx;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;
static int g_autotune = -1;   // -1: read VDWGB_AUTOTUNE once

static bool autotune_on() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_autotune < 0) {
        const char *e = std::getenv("VDWGB_AUTOTUNE");
        g_autotune = (e && e[0] == '1') ? 1 : 0;
    }
    return g_autotune == 1;
}

static int time_stage(vdwgb_data *h, int stage, float &ms) {
    int pre[2 * NKIND];
    for (int s = 0; s < NKIND; ++s) {
        pre[2 * s] = 0;
        pre[2 * s + 1] = h->hsys.tiles[s];
    }
    CK(cudaMemcpy(h->dprefix, pre, sizeof pre, cudaMemcpyHostToDevice), "prefix");
    {
        const int rc = upload_maps(h, true);
        if (rc) return rc;
    }
    CK(cudaMemcpy(h->dsys, &h->hsys, sizeof(SysDev), cudaMemcpyHostToDevice), "descriptor");
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a), "event");
    CK(cudaEventCreate(&b), "event");
    CK(launch_stage(h->ls, h->prec, stage, h->stream), "tune launch");
    CK(cudaEventRecord(a, h->stream), "event");
    for (int r = 0; r < 3; ++r) CK(launch_stage(h->ls, h->prec, stage, h->stream), "tune launch");
    CK(cudaEventRecord(b, h->stream), "event");
    CK(cudaEventSynchronize(b), "event");
    CK(cudaEventElapsedTime(&ms, a, b), "event");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return vdwgb_device_status(h->device);
}

static int apply_tuned(vdwgb_data *h) {
    SysDev &S = h->hsys;
    const TuneKey key{S.nx, S.ny, S.nz, h->prec};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            set_tiles(h, it->second.LZ, it->second.LZi, it->second.Wy, it->second.Wx, it->second.nby, it->second.nbx);
            return 0;
        }
    }
    if (h->alloc_stream || !autotune_on()) return 0;
    // measure on this handle's buffers with a constant density (every point live)
    const int prec = h->prec;
    const size_t N = (size_t)S.nx * S.ny * S.nz;
    const size_t lim = g_dev[h->device].maxsmem - 1024;
    size_t xycap, zcap;
    tile_caps(h->device, prec, xycap, zcap);
    const size_t limxy = std::min(lim, xycap);
    const size_t limz0 = z_stage_cap(0, prec, S.nz, zcap, lim), limz3 = z_stage_cap(3, prec, S.nz, zcap, lim);
    std::vector<double> host(2 * N, 0.0);
    for (size_t i = 0; i < N; ++i) host[i] = 0.01;
    double *tmp = nullptr;
    CK(device_malloc(reinterpret_cast<void **>(&tmp), (4 * N + 1) * sizeof(double)), "tune buffers");
    int rc = 0;
    TuneVal best{S.LZ, S.LZi, S.Wy, S.Wx, h->ls.nbuf[1], h->ls.nbuf[2]};
    auto set_io_dev = [&]() {
        S.n = tmp;
        S.sigma = tmp + N;
        S.dedn = tmp + 2 * N;
        S.dedsigma = tmp + 3 * N;
        S.energy = tmp + 4 * N;
    };
    if (cudaMemcpy(tmp, host.data(), 2 * N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(VDWGB_ECUDA, "tune upload");
    set_io_dev();
    const int cand[8] = {1, 2, 3, 4, 6, 8, 12, 16};
    // z forward first (it writes the records and spectrum the other stages read)
    for (int pass = 0; pass < 4 && !rc; ++pass) {
        if (S.fused && (pass == 1 || pass == 2)) continue;   // y / x run inside the plane kernel
        float best_ms = 1e30f;
        for (int ci = 0; ci < 8 * XY_MAXIN; ++ci) {
            const int c = cand[ci % 8];
            const int nb = 1 + ci / 8;              // x / y passes: input buffers in the ring
            if ((pass == 0 || pass == 3) && ci >= 8) break;
            TuneVal v = best;
            if (pass == 0) {
                if (c > S.nx * S.ny || stage_smem(0, prec, S.nz, c) > limz0) continue;
                v.LZ = c;
            } else if (pass == 1) {
                if (c > S.nzh || stage_smem(1, prec, S.ny, c, nb + (S.sy1 ? 0 : 1)) > limxy) continue;
                v.Wy = c;
                v.nby = nb;
            } else if (pass == 2) {
                if (c > S.nzh || stage_smem(1, prec, S.nx, c, nb + (S.sx1 ? 0 : 1)) > limxy) continue;
                v.Wx = c;
                v.nbx = nb;
            } else {
                if (c > S.nx * S.ny || stage_smem(3, prec, S.nz, c) > limz3) continue;
                v.LZi = c;
            }
            set_tiles(h, v.LZ, v.LZi, v.Wy, v.Wx, v.nby, v.nbx);
            set_io_dev();
            float ms = 0.f;
            const int stage = pass == 0 ? 0 : (pass == 1 ? 2 : (pass == 2 ? 3 : 7));
            rc = time_stage(h, stage, ms);
            if (rc) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
    }
    cudaFree(tmp);
    S.n = S.sigma = nullptr;
    S.dedn = S.dedsigma = S.energy = nullptr;
    if (rc) return rc;
    set_tiles(h, best.LZ, best.LZi, best.Wy, best.Wx, best.nby, best.nbx);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return 0;
}

static int plan(vdwgb_data *h) {
    const int prec = h->prec;
    const int nx = h->nx, ny = h->ny, nz = h->nz, nzh = nz / 2 + 1;
    DevInfo &di = g_dev[h->device];
    SysDev &S = h->hsys;
    std::memset(&S, 0, sizeof S);
    S.nx = nx;
    S.ny = ny;
    S.nz = nz;
    S.nzh = nzh;
    S.yoff = 0;
    S.nyg = ny;
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        if (!factor_axis(dims[a], S.ax[a]))
            return fail(VDWGB_EINVAL, "axis %d length %d: prime factors must be 2, 3, 5, 7", a, dims[a]);
    const size_t lim = di.maxsmem - 1024;
    // in-place x / y transforms (permuted spectrum between the passes) where a
    // two-pass split is compiled (FP32); 0: out of place through the scratch buffer
    S.sx1 = prec == VDWGB_FP32_MIXED ? xy_split(nx) : 0;
    S.sy1 = prec == VDWGB_FP32_MIXED ? xy_split(ny) : 0;
    S.sz1 = prec == VDWGB_FP32_MIXED ? fft_split(nz) : 0;
    const int workx = S.sx1 ? 0 : 1, worky = S.sy1 ? 0 : 1;
    int nbuf = 2;
    size_t xycap, zcap;
    tile_caps(h->device, prec, xycap, zcap);
    choose_tiles(prec, nx, ny, nz, nzh, lim, xycap, zcap, workx, worky, S.LZ, S.LZi, S.Wy, S.Wx, nbuf);
    if (stage_smem(0, prec, nz, S.LZ) > lim || stage_smem(1, prec, nx, S.Wx, nbuf + workx) > lim ||
        stage_smem(1, prec, ny, S.Wy, nbuf + worky) > lim || stage_smem(3, prec, nz, S.LZi) > lim)
        return fail(VDWGB_EINVAL, "grid %dx%dx%d too large for one block per pencil in this precision",
                    nx, ny, nz);
    set_metric(h);
    // half-spectrum k-points sorted by kernel-table interval on the device and
    // cut into chunks (below), or, for the plane kernel, per plane and cluster rank
    const int maxspan = prec == VDWGB_FP32_MIXED ? SPAN32 : SPAN64;
    const int chunkmax = prec == VDWGB_FP32_MIXED ? CHUNK32 : CHUNK64;
    const size_t nk = (size_t)nx * ny * nzh;
    std::vector<unsigned short> kord;
    int maxcl = 0;
    const int C = fused_cluster(h, di.maxsmem - 1024, maxcl);
    S.fused = C;
    size_t nchunk_cap = 0, nepart_cap = 0;
    if (C) {
        build_kord(S, C, kord, S.kstride);
        S.tiles[4] = 0;
        S.tiles[5] = nzh;
        S.nepart = nzh * C;
        nepart_cap = S.nepart;
    } else {
        S.tiles[5] = 0;
        nchunk_cap = max_chunks(nk, chunkmax);
        nepart_cap = nchunk_cap * (prec == VDWGB_FP32_MIXED ? C32_CWARPS : 1);
    }
    // memory
    const size_t nspec = nk * NQ;
    CK(dalloc(h, &h->spec, nspec * elem_bytes(prec)), "work buffer");
    CK(dalloc(h, &h->rec, (size_t)nx * ny * nz * rec_bytes(prec)), "point records");
    CK(dalloc(h, &h->epart, nepart_cap * sizeof(double)), "energy partials");
    if (C) {
        CK(dalloc(h, &h->kord, kord.size() * sizeof(unsigned short)), "plane k-point order");
        CK(dupload(h, h->kord, kord.data(), kord.size() * sizeof(unsigned short)), "plane k-point order");
    } else {
        CK(dalloc(h, &h->kidx, nk * sizeof(unsigned)), "k-point order");
        CK(dalloc(h, &h->chunks, nchunk_cap * sizeof(int4)), "chunks");
    }
    S.kidx = h->kidx;
    S.chunks = h->chunks;
    S.kord = h->kord;
    for (int a = 0; a < 3; ++a) {
        std::vector<double> w = twiddles(dims[a]);
        if (prec == VDWGB_FP32_MIXED) {
            std::vector<float> wf(w.size());
            for (size_t i = 0; i < w.size(); ++i) wf[i] = (float)w[i];
            CK(dalloc(h, &h->tw[a], wf.size() * sizeof(float)), "twiddles");
            CK(dupload(h, h->tw[a], wf.data(), wf.size() * sizeof(float)), "twiddles");
        } else {
            CK(dalloc(h, &h->tw[a], w.size() * sizeof(double)), "twiddles");
            CK(dupload(h, h->tw[a], w.data(), w.size() * sizeof(double)), "twiddles");
        }
        S.tw[a] = h->tw[a];
    }
    S.spec = h->spec;
    S.rec = h->rec;
    S.epart = h->epart;
    S.err = di.err;
    h->bytes = nspec * elem_bytes(prec) + (size_t)nx * ny * nz * rec_bytes(prec) + nepart_cap * sizeof(double) +
               (C ? 0 : nk * sizeof(unsigned)) + nchunk_cap * sizeof(int4) + kord.size() * sizeof(unsigned short);
    CK(dalloc(h, &h->dsys, sizeof(SysDev)), "descriptor");
    CK(dalloc(h, &h->dprefix, 2 * NKIND * sizeof(int)), "prefix");
    if (prec == VDWGB_FP32_MIXED) CK(dalloc(h, &h->tmap, 2 * sizeof(CUtensorMap)), "tensor maps");
    // launch set
    LaunchSet &L = h->ls;
    L.sys = h->dsys;
    L.nsys = 1;
    L.maxspan = maxspan;
    L.err = di.err;
    L.smem[4] = contract_smem(prec, maxspan);
    L.twmax[4] = L.bufelems[4] = L.nbuf[4] = 0;
    L.total[4] = S.tiles[4];
    L.prefix[4] = h->dprefix + 8;
    L.grid[4] = 0;
    L.prefix[5] = h->dprefix + 10;
    L.total[5] = S.tiles[5];
    L.cluster = C;
    L.smem[5] = C ? plane_smem(nx, ny, C) : 0;
    L.grid[5] = C ? (nzh < maxcl ? nzh : maxcl) : 0;       // clusters
    set_tiles(h, S.LZ, S.LZi, S.Wy, S.Wx, nbuf, nbuf);
    TableRefs tr;
    CK(table_get(h->device, tr), "kernel table");
    if (!h->kernel_k.empty()) {
        // the caller's kernel: its own spline coefficients in place of the resident table's
        CK(table_custom(h->kernel_k.data(), h->ktab, h->alloc_stream ? h->alloc_stream : 0), "caller's kernel table");
        tr.cub64 = h->ktab.cub64;
        tr.lin64 = h->ktab.lin64;
        tr.cub32 = h->ktab.cub32;
        tr.lin32 = h->ktab.lin32;
    }
    if (prec == VDWGB_FP32_MIXED)
        L.table = h->interp == VDWGB_INTERP_LINEAR ? (const void *)tr.lin32 : (const void *)tr.cub32;
    else
        L.table = h->interp == VDWGB_INTERP_LINEAR ? (const void *)tr.lin64 : (const void *)tr.cub64;
    h->table = L.table;
    if (!h->alloc_stream) CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
    if (!C) {
        const int rc = sort_kpoints(h, h->alloc_stream ? h->alloc_stream : h->stream);
        if (rc) return rc;
    }
    {
        int rc = apply_tuned(h);          // cached or measured tile choices
        if (rc) return rc;
    }
    return upload_plan(h);
}

static bool axis_ok(int n) {
    if (n < 1 || n > 1024) return false;
    AxisPlan p;
    return factor_axis(n, p);
}

extern "C" {

int vdwgb_new(int functional, vdwgb_handle *out) {
    if (!out) return fail(VDWGB_EINVAL, "null output handle");
    *out = nullptr;
    if (functional != VDWGB_DF1 && functional != VDWGB_DF2)
        return fail(VDWGB_EINVAL, "unknown functional %d", functional);
    vdwgb_data *h = new (std::nothrow) vdwgb_data();
    if (!h) return fail(VDWGB_ENOMEM, "host allocation");
    h->functional = functional;
    *out = h;
    return 0;
}

int vdwgb_set_unit_cell(vdwgb_handle h, int nx, int ny, int nz, double c00, double c01, double c02,
                        double c10, double c11, double c12, double c20, double c21, double c22) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz))
        return fail(VDWGB_EINVAL, "grid %dx%dx%d: each axis 1..1024 with prime factors 2, 3, 5, 7", nx, ny, nz);
    const double c[9] = {c00, c01, c02, c10, c11, c12, c20, c21, c22};
    for (double v : c)
        if (!std::isfinite(v)) return fail(VDWGB_EINVAL, "non-finite cell component");
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    if (!(std::fabs(det) > 1e-12)) return fail(VDWGB_EINVAL, "cell volume is zero");
    if (h->inited) release(h);
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    std::memcpy(h->cell, c, sizeof c);
    h->cell_set = true;
    return 0;
}

int vdwgb_set_kernel_k(vdwgb_handle h, const double *phik) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (h->inited) return fail(VDWGB_ESTATE, "set the kernel table before init");
    if (!phik) {
        h->kernel_k.clear();                 // back to the resident vdW-DF table
        return 0;
    }
    for (size_t i = 0; i < (size_t)NPAIR * NK; ++i)
        if (!std::isfinite(phik[i])) return fail(VDWGB_EINVAL, "kernel table entry %zu is not finite", i);
    h->kernel_k.assign(phik, phik + (size_t)NPAIR * NK);
    return 0;
}

int vdwgb_set_interp(vdwgb_handle h, int interp) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (interp != VDWGB_INTERP_CUBIC && interp != VDWGB_INTERP_LINEAR)
        return fail(VDWGB_EINVAL, "unknown interpolation %d", interp);
    if (h->inited) return fail(VDWGB_ESTATE, "set the interpolation before init");
    h->interp = interp;
    return 0;
}

}  // extern "C"

int vdwgb::handle_init(vdwgb_data *h, int device, int precision, cudaStream_t alloc_stream) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->cell_set) return fail(VDWGB_ESTATE, "set the unit cell before init");
    if (precision != VDWGB_FP64 && precision != VDWGB_FP32_MIXED)
        return fail(VDWGB_EINVAL, "unknown precision %d", precision);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VDWGB_EINVAL, "no CUDA device %d", device);
    if (h->inited) release(h);
    int rc = device_setup(device);
    if (rc) return rc;
    CK(cudaSetDevice(device), "cudaSetDevice");
    h->device = device;
    h->prec = precision;
    h->alloc_stream = alloc_stream;
    rc = plan(h);
    if (rc) {
        release(h);
        return rc;
    }
    if (alloc_stream) {
        const size_t N = (size_t)h->nx * h->ny * h->nz;
        CK(dalloc(h, &h->d_io, (4 * N + 1) * sizeof(double)), "staging");
        h->bytes += (4 * N + 1) * sizeof(double);
    }
    h->inited = true;
    return 0;
}

void vdwgb::handle_release(vdwgb_data *h) { release(h); }

int vdwgb::handle_sort_kpoints(vdwgb_data *h, cudaStream_t st) { return sort_kpoints(h, st); }

int vdwgb::handle_upload_plan(vdwgb_data *h) { return upload_plan(h); }

void vdwgb::handle_use_spec(vdwgb_data *h, void *spec) {
    if (!h->spec_external) dfree(h, h->spec);
    h->spec = spec;
    h->spec_external = true;
    h->hsys.spec = spec;
}

int vdwgb::device_sms(int device) { return (device >= 0 && device < 64) ? g_dev[device].sms : 0; }

int vdwgb::handle_replan(vdwgb_data *h, const double *cell9, int functional) {
    if (!h || !h->inited) return fail(VDWGB_ESTATE, "re-plan of an uninitialised handle");
    if (h->hsys.fused) return fail(VDWGB_ESTATE, "re-plan of a plane-kernel plan");
    // the same cell (repeated evaluations of one system) keeps the k-point
    // order and chunks: they depend on the metric only
    const bool same_cell = std::memcmp(h->cell, cell9, sizeof h->cell) == 0;
    std::memcpy(h->cell, cell9, sizeof h->cell);
    h->functional = functional;
    set_metric(h);
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    if (!same_cell) {
        const int rc = sort_kpoints(h, h->alloc_stream ? h->alloc_stream : h->stream);
        if (rc) return rc;
    }
    return upload_plan(h);
}

size_t vdwgb::handle_io_bytes(const vdwgb_data *h) { return h->bytes; }

extern "C" {

int vdwgb_init_cuda(vdwgb_handle h, int device, int precision) {
    return handle_init(h, device, precision, nullptr);
}

// a descriptor left in the spin-polarised form (q0 given) goes back to the
// plain form, uploaded by the next set_io
static void plain_form(vdwgb_data *h) {
    if (h->hsys.q0in) {
        h->hsys.q0in = 0;
        h->last_ptr[0] = nullptr;
    }
}

static int set_io(vdwgb_data *h, const double *n, const double *s, double *dn, double *ds, double *e,
                  cudaStream_t st) {
    const double *p[5] = {n, s, dn, ds, e};
    if (std::memcmp(p, h->last_ptr, sizeof p) == 0) return 0;
    h->hsys.n = n;
    h->hsys.sigma = s;
    h->hsys.dedn = dn;
    h->hsys.dedsigma = ds;
    h->hsys.energy = e;
    // pageable source: the copy has consumed it when the call returns
    CK(cudaMemcpyAsync(h->dsys, &h->hsys, sizeof(SysDev), cudaMemcpyHostToDevice, st), "descriptor update");
    std::memcpy(h->last_ptr, p, sizeof p);
    return 0;
}

int vdwgb_calculate_device(vdwgb_handle h, const double *d_rho, const double *d_sigma, double *d_dedrho,
                           double *d_dedsigma, double *d_energy, void *cuda_stream) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->inited) return fail(VDWGB_ESTATE, "calculate before init");
    if (!d_rho || !d_sigma || !d_dedrho || !d_dedsigma || !d_energy)
        return fail(VDWGB_EINVAL, "null array");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    plain_form(h);
    int rc = set_io(h, d_rho, d_sigma, d_dedrho, d_dedsigma, d_energy, st);
    if (rc) return rc;
    CK(launch_all(h->ls, h->prec, st), "launch");
    return 0;
}

int vdwgb_calculate(vdwgb_handle h, const double *rho, const double *sigma, double *dedrho, double *dedsigma,
                    double *energy) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->inited) return fail(VDWGB_ESTATE, "calculate before init");
    if (!rho || !sigma || !dedrho || !dedsigma || !energy) return fail(VDWGB_EINVAL, "null array");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->d_io) {
        CK(device_malloc(reinterpret_cast<void **>(&h->d_io), (4 * N + 1) * sizeof(double)), "staging");
        h->bytes += (4 * N + 1) * sizeof(double);
    }
    double *dn = h->d_io, *ds = dn + N, *odn = ds + N, *ods = odn + N, *oe = ods + N;
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(dn, rho, N * sizeof(double), cudaMemcpyHostToDevice, st), "copy rho");
    CK(cudaMemcpyAsync(ds, sigma, N * sizeof(double), cudaMemcpyHostToDevice, st), "copy sigma");
    plain_form(h);
    int rc = set_io(h, dn, ds, odn, ods, oe, st);
    if (rc) return rc;
    CK(launch_all(h->ls, h->prec, st), "launch");
    CK(cudaMemcpyAsync(dedrho, odn, N * sizeof(double), cudaMemcpyDeviceToHost, st), "copy dedrho");
    CK(cudaMemcpyAsync(dedsigma, ods, N * sizeof(double), cudaMemcpyDeviceToHost, st), "copy dedsigma");
    CK(cudaMemcpyAsync(energy, oe, sizeof(double), cudaMemcpyDeviceToHost, st), "copy energy");
    CK(cudaStreamSynchronize(st), "synchronize");
    return vdwgb_device_status(h->device);
}

int vdwgb_device_status(int device) {
    if (device < 0 || device >= 64 || !g_dev[device].ready) return 0;
    int v = 0;
    CK(cudaSetDevice(device), "cudaSetDevice");
    if (take_injection(g_inj_wait)) {
        // as a kernel whose bounded wait ran out leaves it
        const int one = 1;
        CK(cudaMemcpy(g_dev[device].err, &one, sizeof(int), cudaMemcpyHostToDevice), "status injection");
    }
    int flag[2] = {0, 0};
    CK(cudaMemcpy(flag, g_dev[device].err, 2 * sizeof(int), cudaMemcpyDeviceToHost), "status");
    v = flag[0];
    if (v) {
        CK(cudaMemset(g_dev[device].err, 0, 2 * sizeof(int)), "status");
        if (v == 2) return fail(VDWGB_ECUDA, "contraction: a k-point's table interval was outside its chunk's rows");
        if (v == 3)
            return fail(VDWGB_ECUDA, "checked build: an out-of-range access was skipped (check at source line %d)",
                        flag[1]);
        return fail(VDWGB_ETIMEDOUT, "a kernel's bounded wait for its staged tile ran out");
    }
    return 0;
}

double vdwgb_calculate_simple(vdwgb_handle h, const double *rho, const double *sigma, double *dedrho,
                              double *dedsigma) {
    double e = NAN;
    if (vdwgb_calculate(h, rho, sigma, dedrho, dedsigma, &e) != 0) return NAN;
    return e;
}

int vdwgb_finalize(vdwgb_handle *hp) {
    if (!hp) return fail(VDWGB_EINVAL, "null handle pointer");
    if (*hp) {
        release(*hp);
        delete *hp;
    }
    *hp = nullptr;
    return 0;
}

const char *vdwgb_strerror(int code) {
    switch (code) {
        case VDWGB_OK: return "success";
        case VDWGB_EINVAL: return "invalid argument";
        case VDWGB_ENOMEM: return "out of memory";
        case VDWGB_ECUDA: return "CUDA error";
        case VDWGB_ESTATE: return "call out of sequence";
        case VDWGB_ETIMEDOUT: return "timed out";
        case VDWGB_EAGAIN: return "not admitted, retry later";
        case VDWGB_ENOTFOUND: return "unknown request";
        default: return "unknown error";
    }
}

const char *vdwgb_last_error(void) { return g_err.c_str(); }

int vdwgb_print(vdwgb_handle h) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    printf("vdwgb handle: functional vdW-DF%d, interp %s\n", h->functional,
           h->interp == VDWGB_INTERP_LINEAR ? "linear" : "cubic");
    printf("  grid %d x %d x %d, cell rows (%g %g %g) (%g %g %g) (%g %g %g)\n", h->nx, h->ny, h->nz,
           h->cell[0], h->cell[1], h->cell[2], h->cell[3], h->cell[4], h->cell[5], h->cell[6], h->cell[7],
           h->cell[8]);
    if (h->inited) {
        const SysDev &S = h->hsys;
        printf("  device %d, %s, tiles zf %d y %d x %d zi %d chunks %d (LZ %d, LZi %d, Wy %d, Wx %d, nbuf %d), %.1f MB\n",
               h->device, h->prec == VDWGB_FP32_MIXED ? "FP32-mixed" : "FP64", S.tiles[0], S.tiles[1], S.tiles[2],
               S.tiles[3], S.tiles[4], S.LZ, S.LZi, S.Wy, S.Wx, h->ls.nbuf[1], h->bytes / 1e6);
        for (int a = 0; a < 3; ++a) {
            printf("  axis %d n=%d radices", a, S.ax[a].n);
            for (int s = 0; s < S.ax[a].nst; ++s) printf(" %d", S.ax[a].rad[s]);
            printf("\n");
        }
    } else {
        printf("  not initialised\n");
    }
    fflush(stdout);
    return 0;
}

int vdwgb_has_cuda(void) {
    int n = 0;
    return cudaGetDeviceCount(&n) == cudaSuccess && n > 0 ? 1 : 0;
}

size_t vdwgb_footprint_bytes(int nx, int ny, int nz, int precision) {
    const int p = precision == VDWGB_FP32_MIXED ? VDWGB_FP32_MIXED : VDWGB_FP64;
    const size_t nzh = (size_t)nz / 2 + 1;
    const size_t N = (size_t)nx * ny * nz;
    const size_t nk = (size_t)nx * ny * nzh;
    const size_t chunks = max_chunks(nk, p == VDWGB_FP32_MIXED ? CHUNK32 : CHUNK64);
    const size_t parts = chunks * (p == VDWGB_FP32_MIXED ? C32_CWARPS : 1);
    return nk * NQ * elem_bytes(p) + N * rec_bytes(p) + nk * sizeof(unsigned) + chunks * sizeof(int4) +
           parts * sizeof(double);
}

int vdwgb_launches_per_call(vdwgb_handle h) {
    if (!h || !h->inited) return 0;
    return count_launches(h->ls);
}

int vdwgb_kernel_table(int device, double *phik, double *phir, double *qmesh) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VDWGB_EINVAL, "no CUDA device %d", device);
    int rc = device_setup(device);
    if (rc) return rc;
    TableRefs tr;
    CK(table_get(device, tr), "kernel table");
    CK(cudaSetDevice(device), "cudaSetDevice");
    if (phik) CK(cudaMemcpy(phik, tr.phik, (size_t)NPAIR * NK * sizeof(double), cudaMemcpyDeviceToHost), "copy");
    if (phir)
        CK(cudaMemcpy(phir, tr.phir, (size_t)NPAIR * (NR + 1) * sizeof(double), cudaMemcpyDeviceToHost), "copy");
    if (qmesh) {
        QMeshDev q;
        host_qmesh(q);
        std::memcpy(qmesh, q.q, NQ * sizeof(double));
    }
    return 0;
}

int vdwgb_phi(int device, int npts, const double *d1, const double *d2, double *out) {
    if (npts < 0 || (npts > 0 && (!d1 || !d2 || !out))) return fail(VDWGB_EINVAL, "bad arguments");
    if (npts == 0) return 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VDWGB_EINVAL, "no CUDA device %d", device);
    int rc = device_setup(device);
    if (rc) return rc;
    CK(table_phi(device, npts, d1, d2, out), "phi");
    return 0;
}

double vdwgb_table_build_seconds(int device) { return table_seconds(device); }

int vdwgb_inject_fault(int kind, int count) {
    if (count < 0) return fail(VDWGB_EINVAL, "negative injection count");
    switch (kind) {
        case VDWGB_FAULT_NONE:
            g_inj_alloc = 0;
            g_inj_wait = 0;
            return 0;
        case VDWGB_FAULT_ALLOC:
            g_inj_alloc = count;
            return 0;
        case VDWGB_FAULT_WAIT:
            g_inj_wait = count;
            return 0;
        default:
            return fail(VDWGB_EINVAL, "unknown fault kind %d", kind);
    }
}

int vdwgb_set_fused(int enable) {
    std::lock_guard<std::mutex> lk(g_fused_mu);
    g_fused = enable ? 1 : 0;
    return 0;
}

int vdwgb_set_autotune(int enable) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_autotune = enable ? 1 : 0;
    return 0;
}

int vdwgb_set_tiles(vdwgb_handle h, int lz, int lzi, int wy, int wx, int nby, int nbx) {
    if (!h) return fail(VDWGB_EINVAL, "null handle");
    if (!h->inited) return fail(VDWGB_ESTATE, "handle not initialised");
    if (h->nbatch > 0) return fail(VDWGB_ESTATE, "handle is part of a live batch");
    SysDev &S = h->hsys;
    if (S.fused) return fail(VDWGB_ESTATE, "plan uses the plane kernel (no y / x tiles)");
    const int nl = S.nx * S.ny;
    if (lz < 1 || lz > nl || lzi < 1 || lzi > nl || wy < 1 || wy > S.nzh || wx < 1 || wx > S.nzh || nby < 1 ||
        nby > XY_MAXIN || nbx < 1 || nbx > XY_MAXIN)
        return fail(VDWGB_EINVAL, "tile shape out of range");
    const size_t lim = g_dev[h->device].maxsmem - 1024;
    const int workx = S.sx1 ? 0 : 1, worky = S.sy1 ? 0 : 1;
    if (stage_smem(0, h->prec, S.nz, lz) > lim || stage_smem(3, h->prec, S.nz, lzi) > lim ||
        stage_smem(1, h->prec, S.ny, wy, nby + worky) > lim || stage_smem(1, h->prec, S.nx, wx, nbx + workx) > lim)
        return fail(VDWGB_EINVAL, "tile shape exceeds shared memory");
    cudaSetDevice(h->device);
    CK(cudaDeviceSynchronize(), "set tiles: wait for evaluations in flight");
    set_tiles(h, lz, lzi, wy, wx, nby, nbx);
    return upload_plan(h);
}

int vdwgb_plan_info(vdwgb_handle h, int *info) {
    if (!h || !info) return fail(VDWGB_EINVAL, "null argument");
    if (!h->inited) return fail(VDWGB_ESTATE, "handle not initialised");
    const SysDev &S = h->hsys;
    info[0] = S.LZ;
    info[1] = S.LZi;
    info[2] = S.Wy;
    info[3] = S.Wx;
    info[4] = h->ls.nbuf[1] * 10 + h->ls.nbuf[2];
    info[5] = S.tiles[4];
    info[6] = count_launches(h->ls);
    info[8] = S.fused;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    info[7] = g_tune.count(TuneKey{S.nx, S.ny, S.nz, h->prec}) ? 1 : 0;
    return 0;
}

int vdwgb_q0(int device, int precision, int functional, int npts, const double *n, const double *sigma,
             double *q0, double *dq0dn, double *dq0dsigma) {
    if (npts < 0 || (npts > 0 && (!n || !sigma || !q0 || !dq0dn || !dq0dsigma)))
        return fail(VDWGB_EINVAL, "bad arguments");
    if (functional != VDWGB_DF1 && functional != VDWGB_DF2) return fail(VDWGB_EINVAL, "unknown functional");
    if (precision != VDWGB_FP64 && precision != VDWGB_FP32_MIXED) return fail(VDWGB_EINVAL, "unknown precision");
    if (npts == 0) return 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VDWGB_EINVAL, "no CUDA device %d", device);
    int rc = device_setup(device);
    if (rc) return rc;
    CK(cudaSetDevice(device), "cudaSetDevice");
    double *b = nullptr;
    CK(device_malloc(reinterpret_cast<void **>(&b), 5 * (size_t)npts * sizeof(double)), "q0 buffers");
    cudaError_t e = cudaMemcpy(b, n, npts * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + npts, sigma, npts * sizeof(double), cudaMemcpyHostToDevice);
    const double Z = functional == VDWGB_DF2 ? -1.887 : -0.8491;
    if (e == cudaSuccess) e = launch_q0(precision, npts, b, b + npts, Z, b + 2 * npts, b + 3 * npts, b + 4 * npts);
    if (e == cudaSuccess) e = cudaMemcpy(q0, b + 2 * npts, npts * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dq0dn, b + 3 * npts, npts * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dq0dsigma, b + 4 * npts, npts * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(b);
    if (e != cudaSuccess) return cuda_fail(e, "q0");
    return 0;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct vdwgb_batch_s {
    std::vector<vdwgb_data *> hs;
    int device = -1;
    int prec = 0;
    SysDev *dsys = nullptr;
    int *dprefix = nullptr;
    std::vector<SysDev> host;
    LaunchSet ls;
    std::vector<const double *> last;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    bool timing = false;
    std::vector<std::vector<cudaEvent_t>> pending;   // NSTAGE + 1 events per timed call
    std::vector<std::vector<cudaEvent_t>> spare;
    double *d_energy = nullptr;                        // host-pointer path
    cudaStream_t own = nullptr;
    // the batch as parts (systems [pstart[p], pstart[p + 1])) whose stage
    // chains are independent branches (nparts = 0: one launch set for all)
    static constexpr int MAXPARTS = 8;
    int nparts = 0;
    int pstart[MAXPARTS + 1] = {};
    LaunchSet part[MAXPARTS];
    int *dprefix2 = nullptr;
    cudaStream_t capp[MAXPARTS] = {};                  // capture streams of parts 1.. (part 0: cap)
    cudaStream_t hst[MAXPARTS] = {};                   // host-pointer path: one stream per part
    cudaGraph_t hgraph[MAXPARTS] = {};                 // host-pointer path: one stage chain per part
    cudaGraphExec_t hexec[MAXPARTS] = {};
    double *h_energy = nullptr;                        // pinned staging of the energies (the caller's
                                                       // array may be pageable: a copy into it would block)
    cudaEvent_t cev[2 * MAXPARTS] = {};
};

// Parts of a batch: K = VDWGB_BATCH_SPLIT (0 or 1: none; 2..8; default 6:
// measured on 64 uneven grids, the captured graph runs alike with 4, 6 and 8
// parts, and the host-array call leaves the least copy time exposed with 6,
// one part per stream priority level of the GPU)
// capped by the system count; boundary p at the system prefix whose grid
// points come closest to p/K of the total (boundaries strictly increasing).
// Returns the number of parts (0: no split) and fills start[0..parts].
static int batch_parts(vdwgb_data *const *hs, int count, int *start) {
    int K = 6;
    {
        const char *e = std::getenv("VDWGB_BATCH_SPLIT");
        if (e && e[0] >= '0' && e[0] <= '9') K = e[0] - '0';
    }
    if (K > vdwgb_batch_s::MAXPARTS) K = vdwgb_batch_s::MAXPARTS;
    if (K > count) K = count;
    if (K < 2) return 0;
    std::vector<double> acc(count + 1, 0.0);
    for (int i = 0; i < count; ++i) acc[i + 1] = acc[i] + (double)hs[i]->nx * hs[i]->ny * hs[i]->nz;
    start[0] = 0;
    for (int p = 1; p < K; ++p) {
        const double target = acc[count] * p / K;
        int best = start[p - 1] + 1;
        for (int i = best; i <= count - (K - p); ++i)
            if (std::fabs(acc[i] - target) < std::fabs(acc[best] - target)) best = i;
        start[p] = best;
    }
    start[K] = count;
    return K;
}

}  // extern "C"

int vdwgb::batch_launchset(vdwgb_data *const *hs, int count, SysDev *hdesc, int *pre, const SysDev *ddesc,
                           const int *dprefix, LaunchSet &L) {
    std::memset(&L, 0, sizeof L);
    for (int s = 0; s < NKIND; ++s) pre[s * (count + 1)] = 0;   // the caller's array may hold an older launch
    const int device = hs[0]->device;
    const int prec = hs[0]->prec;
    DevInfo &di = g_dev[device];
    const size_t lim = di.maxsmem - 1024;
    // z-inverse: the direct form (nothing staged) is the FP32 one; a batch
    // holds one precision
    const bool zdirect = prec == VDWGB_FP32_MIXED;
    for (int i = 0; i < count; ++i) {
        hdesc[i] = hs[i]->hsys;
        const SysDev &D = hdesc[i];
        for (int s = 0; s < NKIND; ++s) {
            pre[s * (count + 1) + i + 1] = pre[s * (count + 1) + i] + D.tiles[s];
            if (hs[i]->ls.smem[s] > L.smem[s]) L.smem[s] = hs[i]->ls.smem[s];
            if (hs[i]->ls.twmax[s] > L.twmax[s]) L.twmax[s] = hs[i]->ls.twmax[s];
            if (s != 3 && hs[i]->ls.bufelems[s] > L.bufelems[s]) L.bufelems[s] = hs[i]->ls.bufelems[s];
            if (i == 0 || hs[i]->ls.nbuf[s] < L.nbuf[s]) L.nbuf[s] = hs[i]->ls.nbuf[s];
            if (hs[i]->ls.work[s] > L.work[s]) L.work[s] = hs[i]->ls.work[s];
        }
        if (!zdirect) {
            L.bufelems[3] = std::max(L.bufelems[3], D.LZi * D.nzh * NQ);
            L.recelems = std::max(L.recelems, D.LZi * D.nz);
        }
        L.abelems = std::max(L.abelems, D.nz * z_ld(D.LZi));
    }
    L.sys = ddesc;
    L.nsys = count;
    L.err = hs[0]->ls.err;
    L.maxspan = hs[0]->ls.maxspan;
    L.table = hs[0]->table;
    // x / y stages: shared memory from the largest row tile and twiddle table of the batch
    const size_t c = prec == VDWGB_FP32_MIXED ? 8 : 16;
    for (int s = 1; s <= 2; ++s)
        L.smem[s] = xy_smem_bytes(L.twmax[s], L.bufelems[s], L.nbuf[s] + L.work[s], c);
    L.smem[3] = zinv_smem(prec, L.twmax[3], L.bufelems[3], L.recelems, L.abelems, 1 + L.work[3]);
    if (L.smem[1] > lim || L.smem[2] > lim || L.smem[3] > lim)
        return fail(VDWGB_EINVAL, "batch: combined row tiles exceed shared memory");
    for (int s = 0; s < NKIND; ++s) {
        L.prefix[s] = dprefix + s * (count + 1);
        L.total[s] = pre[s * (count + 1) + count];
        const int cap = di.sms * stage_blocks_per_sm(s, prec, L.smem[s]);
        L.grid[s] = L.total[s] < cap ? L.total[s] : cap;
    }
    // plane kernel: one cluster size per launch; grid in clusters
    L.cluster = 0;
    for (int i = 0; i < count; ++i) {
        const int C = hs[i]->hsys.fused;
        if (!C) continue;
        if (L.cluster && C != L.cluster) return fail(VDWGB_EINVAL, "batch: systems need different cluster sizes");
        L.cluster = C;
    }
    L.grid[5] = 0;
    if (L.total[5] > 0) {
        const int m = plane_max_clusters(L.cluster, L.smem[5]);
        if (m < 1) return fail(VDWGB_EINVAL, "batch: plane kernel does not fit (cluster %d, %zu bytes)", L.cluster,
                               L.smem[5]);
        L.grid[5] = L.total[5] < m ? L.total[5] : m;
    }
    return 0;
}

extern "C" {

int vdwgb_batch_new(vdwgb_handle *handles, int count, vdwgb_batch *out) {
    if (!out) return fail(VDWGB_EINVAL, "null output");
    *out = nullptr;
    if (!handles || count < 1) return fail(VDWGB_EINVAL, "empty batch");
    for (int i = 0; i < count; ++i) {
        if (!handles[i] || !handles[i]->inited) return fail(VDWGB_ESTATE, "handle %d not initialised", i);
        if (handles[i]->device != handles[0]->device || handles[i]->prec != handles[0]->prec ||
            handles[i]->table != handles[0]->table)
            return fail(VDWGB_EINVAL, "handle %d: device, precision and interpolation must match", i);
    }
    vdwgb_batch_s *b = new (std::nothrow) vdwgb_batch_s();
    if (!b) return fail(VDWGB_ENOMEM, "host allocation");
    b->hs.assign(handles, handles + count);
    b->device = handles[0]->device;
    b->prec = handles[0]->prec;
    cudaSetDevice(b->device);
    b->host.resize(count);
    std::vector<int> pre(NKIND * (count + 1), 0);
    cudaError_t e = device_malloc(reinterpret_cast<void **>(&b->dsys), count * sizeof(SysDev));
    if (e == cudaSuccess) e = device_malloc(reinterpret_cast<void **>(&b->dprefix), pre.size() * sizeof(int));
    int rc = e == cudaSuccess ? batch_launchset(handles, count, b->host.data(), pre.data(), b->dsys, b->dprefix, b->ls)
                              : cuda_fail(e, "batch setup");
    if (rc == 0) {
        e = cudaMemcpy(b->dprefix, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->dsys, b->host.data(), count * sizeof(SysDev), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch setup");
    }
    int ps[vdwgb_batch_s::MAXPARTS + 1];
    const int np = rc == 0 ? batch_parts(handles, count, ps) : 0;
    if (np > 0) {
        // launch sets of the parts over the same descriptors, own tile prefix sums
        size_t off[vdwgb_batch_s::MAXPARTS + 1];
        off[0] = 0;
        for (int p = 0; p < np; ++p) off[p + 1] = off[p] + (size_t)NKIND * (ps[p + 1] - ps[p] + 1);
        std::vector<int> p2(off[np], 0);
        e = device_malloc(reinterpret_cast<void **>(&b->dprefix2), off[np] * sizeof(int));
        if (e != cudaSuccess) rc = cuda_fail(e, "batch setup");
        for (int p = 0; p < np && rc == 0; ++p)
            rc = batch_launchset(handles + ps[p], ps[p + 1] - ps[p], b->host.data() + ps[p], p2.data() + off[p],
                                 b->dsys + ps[p], b->dprefix2 + off[p], b->part[p]);
        if (rc == 0) {
            e = cudaMemcpy(b->dprefix2, p2.data(), off[np] * sizeof(int), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch setup");
        }
        if (rc == 0) {
            b->nparts = np;
            for (int p = 0; p <= np; ++p) b->pstart[p] = ps[p];
        }
    }
    if (rc) {
        cudaFree(b->dsys);
        cudaFree(b->dprefix);
        cudaFree(b->dprefix2);
        delete b;
        return rc;
    }
    b->last.assign(5 * count, nullptr);
    for (int i = 0; i < count; ++i) ++handles[i]->nbatch;
    *out = b;
    return 0;
}

int vdwgb_batch_calculate_device(vdwgb_batch b, const double *const *d_rho, const double *const *d_sigma,
                                 double *const *d_dedrho, double *const *d_dedsigma, double *d_energy,
                                 void *cuda_stream) {
    if (!b) return fail(VDWGB_EINVAL, "null batch");
    if (!d_rho || !d_sigma || !d_dedrho || !d_dedsigma || !d_energy) return fail(VDWGB_EINVAL, "null array");
    const int n = (int)b->hs.size();
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    bool changed = false;
    for (int i = 0; i < n; ++i) {
        if (!d_rho[i] || !d_sigma[i] || !d_dedrho[i] || !d_dedsigma[i])
            return fail(VDWGB_EINVAL, "null array of system %d", i);
        const double *p[5] = {d_rho[i], d_sigma[i], d_dedrho[i], d_dedsigma[i], d_energy + i};
        for (int k = 0; k < 5; ++k)
            if (b->last[5 * i + k] != p[k]) {
                b->last[5 * i + k] = p[k];
                changed = true;
            }
        SysDev &S = b->host[i];
        S.n = p[0];
        S.sigma = p[1];
        S.dedn = const_cast<double *>(p[2]);
        S.dedsigma = const_cast<double *>(p[3]);
        S.energy = const_cast<double *>(p[4]);
    }
    if (changed)
        CK(cudaMemcpyAsync(b->dsys, b->host.data(), n * sizeof(SysDev), cudaMemcpyHostToDevice, st),
           "descriptor update");
    if (b->timing) {
        // stages launched directly with events between them (no graph)
        std::vector<cudaEvent_t> ev;
        if (!b->spare.empty()) {
            ev = b->spare.back();
            b->spare.pop_back();
        } else {
            ev.resize(NSTAGE + 1);
            for (auto &x : ev) CK(cudaEventCreate(&x), "event");
        }
        CK(launch_all(b->ls, b->prec, st, ev.data()), "launch");
        b->pending.push_back(ev);
        return 0;
    }
    if (!b->exec) {
        // capture the stage launches once; replays read the descriptors above.
        // Split batch: the parts' stage chains are independent branches of
        // the graph, so a compute-bound stage of one part can run beside a
        // memory-bound stage of another
        CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "capture stream");
        const int np = b->nparts;
        for (int p = 1; p < np; ++p) {
            CK(cudaStreamCreateWithFlags(&b->capp[p], cudaStreamNonBlocking), "capture stream");
            CK(cudaEventCreateWithFlags(&b->cev[2 * p], cudaEventDisableTiming), "event");
            CK(cudaEventCreateWithFlags(&b->cev[2 * p + 1], cudaEventDisableTiming), "event");
        }
        CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t le = cudaSuccess;
        if (np) {
            // fork: parts 1.. branch off the capture stream, join at the end
            for (int p = 1; p < np && le == cudaSuccess; ++p) {
                le = cudaEventRecord(b->cev[2 * p], b->cap);
                if (le == cudaSuccess) le = cudaStreamWaitEvent(b->capp[p], b->cev[2 * p], 0);
            }
            for (int k = 0; k < NSTAGE && le == cudaSuccess; ++k)
                for (int p = 0; p < np && le == cudaSuccess; ++p)
                    le = launch_stage(b->part[p], b->prec, k, p ? b->capp[p] : b->cap);
            for (int p = 1; p < np && le == cudaSuccess; ++p) {
                le = cudaEventRecord(b->cev[2 * p + 1], b->capp[p]);
                if (le == cudaSuccess) le = cudaStreamWaitEvent(b->cap, b->cev[2 * p + 1], 0);
            }
        } else {
            le = launch_all(b->ls, b->prec, b->cap);
        }
        cudaError_t ce = cudaStreamEndCapture(b->cap, &b->graph);
        if (le != cudaSuccess) return cuda_fail(le, "capture launch");
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        CK(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate graph");
    }
    CK(cudaGraphLaunch(b->exec, st), "graph launch");
    return 0;
}

int vdwgb_batch_calculate(vdwgb_batch b, const double *const *rho, const double *const *sigma,
                          double *const *dedrho, double *const *dedsigma, double *energy) {
    if (!b) return fail(VDWGB_EINVAL, "null batch");
    if (!rho || !sigma || !dedrho || !dedsigma || !energy) return fail(VDWGB_EINVAL, "null array");
    const int n = (int)b->hs.size();
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    if (!b->own) CK(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking), "stream");
    if (!b->d_energy) CK(device_malloc(reinterpret_cast<void **>(&b->d_energy), n * sizeof(double)), "energies");
    std::vector<const double *> dr(n), dsg(n);
    std::vector<double *> odn(n), ods(n);
    for (int i = 0; i < n; ++i) {
        vdwgb_data *h = b->hs[i];
        if (!rho[i] || !sigma[i] || !dedrho[i] || !dedsigma[i]) return fail(VDWGB_EINVAL, "null array %d", i);
        const size_t N = (size_t)h->nx * h->ny * h->nz;
        if (!h->d_io) {
            CK(device_malloc(reinterpret_cast<void **>(&h->d_io), (4 * N + 1) * sizeof(double)), "staging");
            h->bytes += (4 * N + 1) * sizeof(double);
        }
        double *d = h->d_io;
        dr[i] = d;
        dsg[i] = d + N;
        odn[i] = d + 2 * N;
        ods[i] = d + 3 * N;
    }
    if (b->nparts && !b->timing) {
        // each part on its own stream: its copies in, its stage graph, its
        // copies out; the copies of one part overlap the kernels of the others
        const int np = b->nparts;
        if (!b->hst[np - 1]) {
            // part p at the p-th highest priority: earlier parts get their
            // blocks first and finish first, so their downloads overlap the
            // kernels of the later parts
            int least = 0, greatest = 0;
            CK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range");
            for (int p = 0; p < np; ++p) {
                const int pr = std::max(greatest, std::min(least, greatest + p));
                if (!b->hst[p]) CK(cudaStreamCreateWithPriority(&b->hst[p], cudaStreamNonBlocking, pr), "stream");
            }
        }
        if (!b->h_energy) CK(cudaMallocHost(&b->h_energy, n * sizeof(double)), "pinned energies");
        for (int p = 0; p < np; ++p) {
            if (b->hexec[p]) continue;
            // each part's stage chain captured once (replays read the descriptors)
            CK(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < NSTAGE && le == cudaSuccess; ++k) le = launch_stage(b->part[p], b->prec, k, b->own);
            cudaError_t ce = cudaStreamEndCapture(b->own, &b->hgraph[p]);
            if (le != cudaSuccess) return cuda_fail(le, "capture launch");
            if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
            CK(cudaGraphInstantiate(&b->hexec[p], b->hgraph[p], 0), "instantiate graph");
        }
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            SysDev &S = b->host[i];
            if (S.n != dr[i] || S.sigma != dsg[i] || S.dedn != odn[i] || S.dedsigma != ods[i] ||
                S.energy != b->d_energy + i) {
                S.n = dr[i];
                S.sigma = dsg[i];
                S.dedn = odn[i];
                S.dedsigma = ods[i];
                S.energy = b->d_energy + i;
                changed = true;
            }
        }
        if (changed) {
            // no evaluation of this batch may still read the descriptors
            CK(cudaDeviceSynchronize(), "synchronize");
            CK(cudaMemcpy(b->dsys, b->host.data(), n * sizeof(SysDev), cudaMemcpyHostToDevice), "descriptors");
            for (auto &q : b->last) q = nullptr;   // the graph path re-uploads its own pointers
        }
        for (int p = 0; p < np; ++p) {
            cudaStream_t st = b->hst[p];
            const int lo = b->pstart[p], hi = b->pstart[p + 1];
            for (int i = lo; i < hi; ++i) {
                const size_t N = (size_t)b->hs[i]->nx * b->hs[i]->ny * b->hs[i]->nz;
                CK(cudaMemcpyAsync(const_cast<double *>(dr[i]), rho[i], N * sizeof(double), cudaMemcpyHostToDevice, st),
                   "copy rho");
                CK(cudaMemcpyAsync(const_cast<double *>(dsg[i]), sigma[i], N * sizeof(double), cudaMemcpyHostToDevice,
                                   st),
                   "copy sigma");
            }
            CK(cudaGraphLaunch(b->hexec[p], st), "graph launch");
            for (int i = lo; i < hi; ++i) {
                const size_t N = (size_t)b->hs[i]->nx * b->hs[i]->ny * b->hs[i]->nz;
                CK(cudaMemcpyAsync(dedrho[i], odn[i], N * sizeof(double), cudaMemcpyDeviceToHost, st), "copy dedrho");
                CK(cudaMemcpyAsync(dedsigma[i], ods[i], N * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "copy dedsigma");
            }
            CK(cudaMemcpyAsync(b->h_energy + lo, b->d_energy + lo, (hi - lo) * sizeof(double), cudaMemcpyDeviceToHost,
                               st),
               "copy energy");
        }
        for (int p = 0; p < np; ++p) CK(cudaStreamSynchronize(b->hst[p]), "synchronize");
        std::memcpy(energy, b->h_energy, n * sizeof(double));
        return vdwgb_device_status(b->device);
    }
    for (int i = 0; i < n; ++i) {
        const size_t N = (size_t)b->hs[i]->nx * b->hs[i]->ny * b->hs[i]->nz;
        CK(cudaMemcpyAsync(const_cast<double *>(dr[i]), rho[i], N * sizeof(double), cudaMemcpyHostToDevice, b->own),
           "copy rho");
        CK(cudaMemcpyAsync(const_cast<double *>(dsg[i]), sigma[i], N * sizeof(double), cudaMemcpyHostToDevice, b->own),
           "copy sigma");
    }
    int rc = vdwgb_batch_calculate_device(b, dr.data(), dsg.data(), odn.data(), ods.data(), b->d_energy, b->own);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        vdwgb_data *h = b->hs[i];
        const size_t N = (size_t)h->nx * h->ny * h->nz;
        CK(cudaMemcpyAsync(dedrho[i], odn[i], N * sizeof(double), cudaMemcpyDeviceToHost, b->own), "copy dedrho");
        CK(cudaMemcpyAsync(dedsigma[i], ods[i], N * sizeof(double), cudaMemcpyDeviceToHost, b->own),
           "copy dedsigma");
    }
    CK(cudaMemcpyAsync(energy, b->d_energy, n * sizeof(double), cudaMemcpyDeviceToHost, b->own), "copy energy");
    CK(cudaStreamSynchronize(b->own), "synchronize");
    return vdwgb_device_status(b->device);
}

int vdwgb_batch_set_timing(vdwgb_batch b, int enable) {
    if (!b) return fail(VDWGB_EINVAL, "null batch");
    b->timing = enable != 0;
    return 0;
}

int vdwgb_batch_stage_ms(vdwgb_batch b, double *ms, int *ncalls) {
    if (!b || !ms) return fail(VDWGB_EINVAL, "null argument");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    for (int k = 0; k < NSTAGE; ++k) ms[k] = 0.0;
    for (auto &ev : b->pending) {
        CK(cudaEventSynchronize(ev[NSTAGE]), "event sync");
        for (int k = 0; k < NSTAGE; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]), "elapsed");
            ms[k] += t;
        }
        b->spare.push_back(ev);
    }
    if (ncalls) *ncalls = (int)b->pending.size();
    b->pending.clear();
    return 0;
}

int vdwgb_batch_launches(vdwgb_batch b) {
    if (!b) return 0;
    if (b->nparts) {
        int total = 0;
        for (int p = 0; p < b->nparts; ++p) total += count_launches(b->part[p]);
        return total;
    }
    return count_launches(b->ls);
}

const char *vdwgb_stage_name(int i) { return stage_name(i); }

int vdwgb_num_stages(void) { return NSTAGE; }

int vdwgb_batch_free(vdwgb_batch *bp) {
    if (!bp) return fail(VDWGB_EINVAL, "null batch pointer");
    vdwgb_batch_s *b = *bp;
    if (b) {
        cudaSetDevice(b->device);
        for (vdwgb_data *h : b->hs) --h->nbatch;
        if (b->exec) cudaGraphExecDestroy(b->exec);
        for (auto &v : b->pending)
            for (auto e : v) cudaEventDestroy(e);
        for (auto &v : b->spare)
            for (auto e : v) cudaEventDestroy(e);
        if (b->own) cudaStreamDestroy(b->own);
        if (b->h_energy) cudaFreeHost(b->h_energy);
        for (int p = 0; p < vdwgb_batch_s::MAXPARTS; ++p) {
            if (b->hst[p]) cudaStreamDestroy(b->hst[p]);
            if (b->capp[p]) cudaStreamDestroy(b->capp[p]);
            if (b->hexec[p]) cudaGraphExecDestroy(b->hexec[p]);
            if (b->hgraph[p]) cudaGraphDestroy(b->hgraph[p]);
        }
        cudaFree(b->d_energy);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->cap) cudaStreamDestroy(b->cap);
        for (auto ev : b->cev)
            if (ev) cudaEventDestroy(ev);
        cudaFree(b->dsys);
        cudaFree(b->dprefix);
        cudaFree(b->dprefix2);
        delete b;
    }
    *bp = nullptr;
    return 0;
}

}  // extern "C"

int vdwgb::handle_set_io(vdwgb_data *h, const double *n, const double *s, double *dn, double *ds, double *e,
                         cudaStream_t st) {
    return set_io(h, n, s, dn, ds, e, st);
}
