// Slab decomposition of one system over P ranks (one GPU each), the
// GPU-side stages of the parallel layout the paper builds on FFTW-MPI (Sec.
// 3, parallelisation): rank r owns the x-planes [r nx/P, (r+1) nx/P) of the
// real-space grid and the y positions [r ny/P, (r+1) ny/P) of the spectrum.
//
//   forward   (x-slab)  q0, theta, transforms along z and y      -> A spectrum
//   pack      A spectrum [xl][d][run] -> send buffer [d][xl][run]
//   all-to-all (the caller's collective): send buffer -> B spectrum of every rank
//   contract  (ky-slab) transforms along x, kernel contraction with the
//             global frequencies of the slab's k-points, energy partial of
//             the rank (the caller sums the ranks' partials), inverse x
//   all-to-all back (the caller's): B spectrum -> receive buffer
//   unpack    receive buffer [d][xl][run] -> A spectrum
//   inverse   (x-slab)  inverse transforms along y and z, potential
//
// run = (ny/P) (nz/2+1) 20 complex values; the receive side of the forward
// exchange needs no unpacking: [s][xl][run] is the ky-slab's [x][yl][kz][a].
// Two handles carry the plan: A on the x-slab grid (nx/P, ny, nz), B on the
// ky-slab grid (nx, ny/P, nz) with the y offset and global y axis that its
// contraction and k-point order use; both normalise with the global grid.
// The work buffers of both are the caller's (device memory the collective
// library can address).
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"
#include "fftreg.cuh"

using namespace vdwgb;

struct vdwgb_slab_s {
    vdwgb_data *A = nullptr, *B = nullptr;
    int P = 1, rank = 0, nx = 0, ny = 0, nz = 0, nxl = 0, nyl = 0, prec = 0, device = 0;
    size_t run_bytes = 0;
};

static size_t slab_elem_bytes(int prec) { return prec == VDWGB_FP32_MIXED ? 8 : 16; }

extern "C" {

size_t vdwgb_slab_bytes(int nx, int ny, int nz, int P, int precision) {
    if (P < 1 || nx < 1 || ny < 1 || nz < 1 || nx % P || ny % P) return 0;
    return (size_t)(nx / P) * ny * (nz / 2 + 1) * NQ * slab_elem_bytes(precision);
}

int vdwgb_slab_free(vdwgb_slab *sp) {
    if (!sp) return fail(VDWGB_EINVAL, "null slab pointer");
    vdwgb_slab_s *s = *sp;
    if (s) {
        if (s->A) vdwgb_finalize(&s->A);
        if (s->B) vdwgb_finalize(&s->B);
        delete s;
    }
    *sp = nullptr;
    return 0;
}

int vdwgb_slab_new(int functional, int nx, int ny, int nz, const double *cell9, int P, int rank, int device,
                   int precision, void *d_aspec, void *d_bspec, vdwgb_slab *out) {
    if (!out) return fail(VDWGB_EINVAL, "null output");
    *out = nullptr;
    if (!cell9 || !d_aspec || !d_bspec) return fail(VDWGB_EINVAL, "null argument");
    if (P < 1 || rank < 0 || rank >= P) return fail(VDWGB_EINVAL, "rank %d of %d", rank, P);
    if (nx < 1 || ny < 1 || nz < 1 || nx % P || ny % P)
        return fail(VDWGB_EINVAL, "grid %dx%dx%d: nx and ny must be multiples of the %d ranks", nx, ny, nz, P);
    if ((reinterpret_cast<uintptr_t>(d_aspec) | reinterpret_cast<uintptr_t>(d_bspec)) & 255)
        return fail(VDWGB_EINVAL, "work buffers must be 256-byte aligned");
    vdwgb_slab_s *s = new (std::nothrow) vdwgb_slab_s();
    if (!s) return fail(VDWGB_ENOMEM, "host allocation");
    s->P = P;
    s->rank = rank;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->nxl = nx / P;
    s->nyl = ny / P;
    s->prec = precision;
    s->device = device;
    s->run_bytes = (size_t)s->nyl * (nz / 2 + 1) * NQ * slab_elem_bytes(precision);
    const double *c = cell9;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    const double N = (double)nx * ny * nz;
    int rc = vdwgb_new(functional, &s->A);
    if (!rc) rc = vdwgb_new(functional, &s->B);
    if (!rc)
        rc = vdwgb_set_unit_cell(s->A, s->nxl, ny, nz, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8]);
    if (!rc)
        rc = vdwgb_set_unit_cell(s->B, nx, s->nyl, nz, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8]);
    if (!rc) rc = vdwgb_init_cuda(s->A, device, precision);
    if (!rc) rc = vdwgb_init_cuda(s->B, device, precision);
    if (!rc && (s->A->hsys.fused || s->B->hsys.fused)) rc = fail(VDWGB_ESTATE, "slabs need the plane kernel off");
    if (rc) {
        vdwgb_slab_free(&s);
        return rc;
    }
    // A: z and y passes of the x-slab (q0, theta, records, potential); the
    // inverse transform normalises by the global point count
    {
        SysDev &S = s->A->hsys;
        LaunchSet &L = s->A->ls;
        S.invN = 1.0 / N;
        S.invNf = (float)S.invN;
        S.escale = 0.5 * std::fabs(det) / (N * N);
        S.tiles[2] = S.tiles[4] = 0;
        L.total[2] = L.total[4] = 0;
        handle_use_spec(s->A, d_aspec);
    }
    // B: x passes and the contraction of the ky-slab: global y frequencies,
    // global energy normalisation, the k-point order of those frequencies
    {
        SysDev &S = s->B->hsys;
        LaunchSet &L = s->B->ls;
        S.yoff = rank * s->nyl;
        S.nyg = ny;
        S.sy1 = precision == VDWGB_FP32_MIXED ? xy_split(ny) : 0;    // the y pass's output order
        S.invN = 1.0 / N;
        S.invNf = (float)S.invN;
        S.escale = 0.5 * std::fabs(det) / (N * N);
        S.tiles[0] = S.tiles[1] = S.tiles[3] = 0;
        L.total[0] = L.total[1] = L.total[3] = 0;
        handle_use_spec(s->B, d_bspec);
        cudaSetDevice(device);
        rc = handle_sort_kpoints(s->B, s->B->stream);
    }
    if (!rc) rc = handle_upload_plan(s->A);
    if (!rc) rc = handle_upload_plan(s->B);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = fail(VDWGB_ECUDA, "slab set-up");
    if (rc) {
        vdwgb_slab_free(&s);
        return rc;
    }
    *out = s;
    return 0;
}

static cudaError_t launch_stages(vdwgb_data *h, const int *stages, int n, cudaStream_t st) {
    for (int i = 0; i < n; ++i) {
        const cudaError_t e = launch_stage(h->ls, h->prec, stages[i], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int vdwgb_slab_forward(vdwgb_slab s, const double *d_rho, const double *d_sigma, void *cuda_stream) {
    if (!s || !d_rho || !d_sigma) return fail(VDWGB_EINVAL, "null argument");
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const vdwgb_data *A = s->A;
    int rc = handle_set_io(s->A, d_rho, d_sigma, A->hsys.dedn, A->hsys.dedsigma, A->hsys.energy, st);
    if (rc) return rc;
    static const int stages[2] = {0, 2};   // z forward (q0, theta), y forward
    const cudaError_t e = launch_stages(s->A, stages, 2, st);
    return e == cudaSuccess ? 0 : cuda_fail(e, "slab forward");
}

int vdwgb_slab_pack(vdwgb_slab s, void *d_send, void *cuda_stream) {
    if (!s || !d_send) return fail(VDWGB_EINVAL, "null argument");
    cudaSetDevice(s->device);
    const cudaError_t e = launch_slab_transpose(s->A->spec, d_send, s->nxl, s->P, s->run_bytes, true,
                                                device_sms(s->device), (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? 0 : cuda_fail(e, "slab pack");
}

int vdwgb_slab_contract(vdwgb_slab s, double *d_energy, void *cuda_stream) {
    if (!s || !d_energy) return fail(VDWGB_EINVAL, "null argument");
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const vdwgb_data *B = s->B;
    int rc = handle_set_io(s->B, B->hsys.n, B->hsys.sigma, B->hsys.dedn, B->hsys.dedsigma, d_energy, st);
    if (rc) return rc;
    static const int stages[4] = {3, 4, 5, 8};   // x forward, contraction, x inverse, energy finish
    const cudaError_t e = launch_stages(s->B, stages, 4, st);
    return e == cudaSuccess ? 0 : cuda_fail(e, "slab contraction");
}

int vdwgb_slab_unpack(vdwgb_slab s, const void *d_recv, void *cuda_stream) {
    if (!s || !d_recv) return fail(VDWGB_EINVAL, "null argument");
    cudaSetDevice(s->device);
    const cudaError_t e = launch_slab_transpose(d_recv, s->A->spec, s->nxl, s->P, s->run_bytes, false,
                                                device_sms(s->device), (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? 0 : cuda_fail(e, "slab unpack");
}

int vdwgb_slab_inverse(vdwgb_slab s, double *d_dedrho, double *d_dedsigma, void *cuda_stream) {
    if (!s || !d_dedrho || !d_dedsigma) return fail(VDWGB_EINVAL, "null argument");
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const vdwgb_data *A = s->A;
    int rc = handle_set_io(s->A, A->hsys.n, A->hsys.sigma, d_dedrho, d_dedsigma, A->hsys.energy, st);
    if (rc) return rc;
    static const int stages[2] = {6, 7};   // y inverse, z inverse (potential)
    const cudaError_t e = launch_stages(s->A, stages, 2, st);
    return e == cudaSuccess ? 0 : cuda_fail(e, "slab inverse");
}

}  // extern "C"
