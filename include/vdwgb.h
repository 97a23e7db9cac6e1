/*
 * vdwgb -- GB300-native vdW-DF nonlocal correlation (Roman-Perez--Soler FFT
 * evaluation of E_c^nl and its potential), arXiv:1703.06999.
 *
 * C ABI.  Plain pointers and sizes only.  Every function returns 0 on
 * success or a negative VDWGB_E* code; nothing is thrown across the ABI.
 * vdwgb_strerror() names a code; vdwgb_last_error() gives the message of the
 * calling thread's last failure.
 *
 * Calling sequence (Sec. 6 of the paper, "The library"): create a handle for
 * a functional (vdwgb_new), give it the grid and unit cell
 * (vdwgb_set_unit_cell), initialise the backend and its memory
 * (vdwgb_init_cuda), evaluate any number of times (vdwgb_calculate /
 * vdwgb_calculate_device), release (vdwgb_finalize).
 *
 * Arrays: row-major [nx][ny][nz], z contiguous (the density grid of Sec. 3
 * with x least contiguous).  Units: bohr and Hartree.  Cell: three rows, the
 * lattice vectors a_1, a_2, a_3 (row i = a_i).
 *
 * Outputs (Eq. dedn, Eq. dedsigma): dedrho[i] = dE/dn(r_i) at fixed sigma and
 * dedsigma[i] = dE/dsigma(r_i) at fixed n, both per unit volume (so that
 * dE = sum_i dV (dedrho_i dn_i + dedsigma_i dsigma_i)).  They are OVERWRITTEN,
 * not accumulated.  Points with n <= 1e-12 give theta = 0 and zero
 * derivatives; sigma < 0 is treated as 0.
 */
#ifndef VDWGB_H
#define VDWGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Functionals: the nonlocal part differs only by Z_ab (appendix, q0):
 * vdW-DF1 Z_ab = -0.8491, vdW-DF2 Z_ab = -1.887. */
enum { VDWGB_DF1 = 1, VDWGB_DF2 = 2 };

/* Precision of the evaluation.
 *   VDWGB_FP64        every step in FP64 (the paper computes in double
 *                     precision, Sec. 6).
 *   VDWGB_FP32_MIXED  theta fields, FFTs and kernel contraction in FP32;
 *                     q0 and the saturation in double-float (pairs of FP32,
 *                     about 46 significant bits: the GPU's FP64 rate is
 *                     1/64 of its FP32 rate); energy partials summed with
 *                     compensated (error-free) sums in a fixed order. */
enum { VDWGB_FP64 = 0, VDWGB_FP32_MIXED = 1 };

/* Kernel interpolation in |k| (Sec. 3, procedure step 3a): the paper
 * interpolates the tabulated phi_ab(k) linearly; the default here is a
 * natural cubic spline through the same table. */
enum { VDWGB_INTERP_CUBIC = 0, VDWGB_INTERP_LINEAR = 1 };

/* Error codes. */
enum {
    VDWGB_OK = 0,
    VDWGB_EINVAL = -1,    /* bad argument (null pointer, bad size or enum)  */
    VDWGB_ENOMEM = -2,    /* device or host allocation failed               */
    VDWGB_ECUDA = -3,     /* a CUDA call failed (message in last_error)     */
    VDWGB_ESTATE = -4,    /* call out of sequence (e.g. calculate before init) */
    VDWGB_ETIMEDOUT = -5, /* a bounded wait ran out                         */
    VDWGB_EAGAIN = -6,    /* not admitted now (serving); retry later        */
    VDWGB_ENOTFOUND = -7  /* unknown request id (serving)                   */
};

typedef struct vdwgb_data *vdwgb_handle;

/* ---- single-system interface (paper-shaped) -------------------------- */

/* Create an empty handle for a functional (cf. vdwxc_new, Sec. 6).
 * functional: VDWGB_DF1 or VDWGB_DF2.  *out receives the handle, owned by
 * the library until vdwgb_finalize.  EINVAL on a bad functional or null out. */
int vdwgb_new(int functional, vdwgb_handle *out);

/* Grid points per axis and the unit cell (cf. vdwxc_set_unit_cell, Sec. 6).
 * nx, ny, nz >= 1 with every prime factor in {2, 3, 5, 7} and each <= 1024
 * (EINVAL otherwise); cXY = component Y of lattice vector X (bohr).  The cell
 * must have positive volume.  Calling it again after init re-plans at the
 * next vdwgb_init_cuda. */
int vdwgb_set_unit_cell(vdwgb_handle h, int nx, int ny, int nz,
                        double c00, double c01, double c02,
                        double c10, double c11, double c12,
                        double c20, double c21, double c22);

/* A caller's convolution kernel in place of the vdW-DF one, before init (the
 * paper's outlook, Sec. 7: the spline decomposition serves any nonlocal
 * functional expressible as a convolution; Sec. 2 end: the kernel enters
 * only as the 20 x 20 radial functions phi_ab(k)).  phik: host array of
 * 210 x 1024 doubles, phik[p * 1024 + j] = phi_ab(k_j) for the symmetric
 * pairs p = (a <= b) in row-major order (a = 0: b = 0..19, then a = 1, ...)
 * on k_j = j 2 pi / 100 bohr^-1; phi is taken as 0 beyond the last point.
 * The q-mesh, theta = n p_a(q0) and q0 stay those of the handle's functional
 * (the mesh values are returned by vdwgb_kernel_table).  The handle builds
 * its own spline coefficients from phik at init (about 20 MB on the device,
 * not counted by vdwgb_footprint_bytes); handles with different tables do
 * not batch together.  NULL restores the vdW-DF table.  EINVAL on a
 * non-finite entry, ESTATE after init. */
int vdwgb_set_kernel_k(vdwgb_handle h, const double *phik);

/* Choose kernel interpolation (VDWGB_INTERP_*) before init.  Default cubic. */
int vdwgb_set_interp(vdwgb_handle h, int interp);

/* Initialise on a CUDA device (cf. vdwxc_init_serial, Sec. 6): builds the
 * resident kernel table on that device (once per device and process),
 * plans the FFTs, allocates the work buffer (20 complex fields on the
 * half spectrum) and the per-point records.  precision: VDWGB_FP64 or
 * VDWGB_FP32_MIXED.  ENOMEM if the device is out of memory, ECUDA on other
 * CUDA failures, ESTATE if the cell was not set. */
int vdwgb_init_cuda(vdwgb_handle h, int device, int precision);

/* Evaluate E_c^nl and its partial derivatives from HOST arrays (cf.
 * vdwxc_calculate, Sec. 6).  rho, sigma: nx*ny*nz doubles (read).  dedrho,
 * dedsigma: nx*ny*nz doubles (overwritten).  energy: one double (written,
 * Hartree).  Blocking; the arrays are copied to and from device staging
 * buffers owned by the handle (page-locked caller memory copies fastest).
 * Callable any number of times after init. */
int vdwgb_calculate(vdwgb_handle h, const double *rho, const double *sigma,
                    double *dedrho, double *dedsigma, double *energy);

/* The same with DEVICE pointers, enqueued on cuda_stream (a cudaStream_t,
 * NULL = the legacy default stream); returns without waiting.  d_energy is
 * one device double.  The caller keeps every pointer valid until the stream
 * work completes and must not run two calls of one handle concurrently. */
int vdwgb_calculate_device(vdwgb_handle h, const double *d_rho, const double *d_sigma,
                           double *d_dedrho, double *d_dedsigma, double *d_energy,
                           void *cuda_stream);

/* Spin-polarised form (svdW-DF: announced in Sec. 1 and the outlook, defined
 * by Thonhauser et al., PRL 115, 136402 (2015)).  Inputs: the two spin
 * densities n_up, n_dn and the same-spin gradient products sigma_upup =
 * |grad n_up|^2, sigma_dndn = |grad n_dn|^2 (the energy does not depend on
 * grad n_up . grad n_dn), [nx][ny][nz] as above.  theta uses the total
 * density n_up + n_dn with the same kernel; q0 takes spin-scaled exchange
 * (each channel with the gradient correction of its doubled density) and
 * PW92 correlation with its spin interpolation, formed in FP64 (FP64 form)
 * or double-float, about 46 bits (FP32-mixed form).  Outputs, OVERWRITTEN,
 * per unit volume: dE/dn_up, dE/dn_dn, dE/dsigma_upup, dE/dsigma_dndn, and
 * the energy.  n_s < 0 and sigma_ss < 0
 * count as 0; points with n_up + n_dn <= 1e-12 give zero outputs; a channel
 * with n_s <= 1e-12 has no exchange term.  The handle allocates 48 bytes
 * per grid point at the first call (64 more for the host form's staging).
 * Host form: blocking, like vdwgb_calculate.  Device form: enqueued on
 * cuda_stream like vdwgb_calculate_device, same rules; ESTATE with the plane
 * kernel on. */
int vdwgb_calculate_spin(vdwgb_handle h, const double *rho_up, const double *rho_dn,
                         const double *sigma_upup, const double *sigma_dndn, double *dedrho_up,
                         double *dedrho_dn, double *dedsigma_upup, double *dedsigma_dndn, double *energy);
int vdwgb_calculate_spin_device(vdwgb_handle h, const double *d_rho_up, const double *d_rho_dn,
                                const double *d_sigma_upup, const double *d_sigma_dndn, double *d_dedrho_up,
                                double *d_dedrho_dn, double *d_dedsigma_upup, double *d_dedsigma_dndn,
                                double *d_energy, void *cuda_stream);

/* Paper-shaped convenience: returns the energy, NaN on any error. */
double vdwgb_calculate_simple(vdwgb_handle h, const double *rho, const double *sigma,
                              double *dedrho, double *dedsigma);

/* Release every resource of the handle and set *h = NULL (cf. vdwxc_finalize). */
int vdwgb_finalize(vdwgb_handle *h);

/* ---- information --------------------------------------------------- */

const char *vdwgb_strerror(int code);
const char *vdwgb_last_error(void);
/* Print the handle's state (functional, grid, cell, plan, memory) to stdout. */
int vdwgb_print(vdwgb_handle h);
/* 1 if a CUDA device is usable by this library, else 0. */
int vdwgb_has_cuda(void);
/* Bytes of device memory one handle of this grid and precision allocates
 * (work buffer + records + partials), excluding the shared kernel table. */
size_t vdwgb_footprint_bytes(int nx, int ny, int nz, int precision);

/* 0, or VDWGB_ETIMEDOUT if a kernel on `device` gave up a bounded wait for
 * its staged data since the last call, or VDWGB_ECUDA if the FP32
 * contraction met a k-point outside the table rows staged for its chunk (an
 * internal invariant: host and device sort k-points with the same FP32
 * arithmetic); the results are then invalid.  The flag is cleared.  The
 * host-array calls check it themselves; callers of the device-pointer calls
 * check it after synchronising. */
int vdwgb_device_status(int device);

/* Number of our kernel launches one evaluation enqueues (stages without
 * work for this handle are not launched). */
int vdwgb_launches_per_call(vdwgb_handle h);

/* Measured arithmetic peak of the CUDA cores of `device` (the paper has no
 * counterpart; this is the denominator of the ALU rooflines of the FP32
 * stage kernels and of the FP64 form).  kind 0: scalar FP32 fused
 * multiply-add; 1: two-lane FP32 fused multiply-add (fma.rn.f32x2, the form
 * the FP32 contraction uses); 2: FP64 fused multiply-add.  *gflops receives
 * 2 x (fused multiply-adds per second) / 1e9 from CUDA events around one
 * launch of eight independent FMA chains per thread, eight 256-thread blocks
 * per SM, after a warm-up launch (about 10 ms each).  Allocates 4 bytes of
 * device memory for the duration of the call.  EINVAL for another kind or
 * device. */
int vdwgb_alu_peak(int device, int kind, double *gflops);

/* ---- kernel table (setup, resident per device) ------------------------ */

/* Copy the resident FP64 tables of `device` to host memory (building them if
 * needed).  phik: 210 * 1024 doubles, phi_ab(k_j) for the symmetric pairs
 * (a <= b, row-major) at k_j = j * 2 pi / 100 bohr; phir: 210 * 1025 doubles,
 * phi_ab(r_i) = phi(q_a r_i, q_b r_i) at r_i = i * 100/1024 bohr; qmesh: 20
 * doubles.  Any pointer may be NULL.  (Sec. 2: the M x M radial functions
 * phi_ab(k) on a discrete k-grid; the kernel phi of Eq. 2.) */
int vdwgb_kernel_table(int device, double *phik, double *phir, double *qmesh);

/* phi(d1[i], d2[i]) for npts pairs on `device` with the table's quadrature
 * (host arrays in and out), for checking the kernel itself. */
int vdwgb_phi(int device, int npts, const double *d1, const double *d2, double *out);

/* q0(n, sigma) and its partial derivatives (appendix, q0 with PW92
 * correlation and the saturation h_5) exactly as the given precision form
 * evaluates them inside vdwgb_calculate (FP64 values either way; the
 * FP32-mixed form evaluates q0 and its derivatives in double-float
 * arithmetic, pairs of FP32 with about 46 significant bits, and rounds the
 * derivatives to FP32).  Host
 * arrays of npts doubles. */
int vdwgb_q0(int device, int precision, int functional, int npts, const double *n, const double *sigma,
             double *q0, double *dq0dn, double *dq0dsigma);

/* Fault injection for testing the error paths without a GPU fault (off by
 * default; the paper has no counterpart).  kind VDWGB_FAULT_ALLOC: the next
 * `count` device allocations the library makes (handle plans, batches,
 * server requests and slots) fail as if the device were out of memory, so
 * the call that needed them returns VDWGB_ENOMEM.  kind VDWGB_FAULT_WAIT: the
 * next `count` calls of vdwgb_device_status (made by the host-array calls,
 * the batch host-array call and the server after each batch) first set the
 * device's status flag, as a kernel whose bounded wait ran out leaves it, so
 * they report VDWGB_ETIMEDOUT.  kind VDWGB_FAULT_NONE disarms both.  EINVAL
 * for another kind or a negative count.  Process-wide, thread-safe. */
enum { VDWGB_FAULT_NONE = 0, VDWGB_FAULT_ALLOC = 1, VDWGB_FAULT_WAIT = 2 };
int vdwgb_inject_fault(int kind, int count);

/* Plane kernel on (1) or off (0, default) for handles initialised after the
 * call.  On: FP32-mixed handles whose x and y lengths are multiples of 16
 * with a compiled two-pass split (16..256) and whose kz-plane fits the shared
 * memory of a 16-CTA cluster run the y transforms, x transforms, kernel
 * contraction and inverses of each kz-plane in one cluster (one HBM round trip
 * of the work buffer instead of five; experimental: slower than the separate
 * passes on 96^3 grids).  Off: separate y, x and contraction passes for every
 * handle.  The environment variable VDWGB_FUSED=1 sets the default to on.
 * Results agree within FP32 rounding either way. */
int vdwgb_set_fused(int enable);

/* Autotuning of tile shapes: when enabled (here or by the environment
 * variable VDWGB_AUTOTUNE=1), vdwgb_init_cuda times every stage kernel for
 * each candidate tile shape that fits shared memory (z-forward lines, y / x
 * kz-columns with 1 to 4 ring buffers, z-inverse lines) on the handle's
 * own buffers and keeps the
 * fastest; the choice is cached per (grid, precision) for the process and
 * reused by later handles, batches and the server.  Default off.  Candidates
 * (and the untuned default) of the FP32-mixed form are capped in shared
 * memory per block: y / x tiles at half of an SM's shared memory less 2.5 KB
 * (two blocks per SM), z tiles at a third less 1.8 KB (three blocks) unless
 * that leaves tiles of a single line.  The environment variables
 * VDWGB_XY_CAP and VDWGB_Z_CAP (bytes), read once per process, replace the
 * two caps. */
int vdwgb_set_autotune(int enable);

/* Replace the tile shapes of an initialised handle's plan (as the autotuner
 * does): z-forward lines per tile lz, z-inverse lines lzi, y / x pass
 * kz-columns wy / wx, and input buffers in the ring of the y / x passes
 * nby / nbx (1..4; 1: no prefetch).  Waits for all work on the device first;
 * call it with no evaluation of this handle in flight.  Returns VDWGB_EINVAL
 * for a shape out of range (lines 1..nx*ny, columns 1..nz/2+1) or beyond
 * shared memory, VDWGB_ESTATE for an uninitialised handle, a handle that a
 * live batch holds (free the batch first) or a plane-kernel plan. */
int vdwgb_set_tiles(vdwgb_handle h, int lz, int lzi, int wy, int wx, int nby, int nbx);

/* Plan of an initialised handle: info[0..8] = z-forward lines per tile,
 * z-inverse lines per tile, y-pass kz-columns, x-pass kz-columns,
 * input buffers in the ring of the y and x passes as 10 * y + x (1: no
 * prefetch, n: n - 1 tiles requested ahead),
 * contraction chunks, kernel launches per evaluation, 1 if the tile shapes
 * were autotuned, cluster size of the plane kernel (0: separate passes). */
int vdwgb_plan_info(vdwgb_handle h, int *info);

/* Seconds spent building the table on `device` (0 if not built). */
double vdwgb_table_build_seconds(int device);

/* ---- batched form: many independent systems, one launch per stage and part */

typedef struct vdwgb_batch_s *vdwgb_batch;

/* Create a batch of `count` initialised handles (same device and precision,
 * any grids).  The batch owns a launch plan over all systems, one per part
 * (see vdwgb_batch_launches), and a CUDA graph of their stages; the handles
 * stay owned by the caller and must outlive the batch.  While a batch holds
 * a handle, vdwgb_set_tiles refuses it. */
int vdwgb_batch_new(vdwgb_handle *handles, int count, vdwgb_batch *out);

/* Evaluate every system of the batch from DEVICE arrays enqueued on
 * cuda_stream: d_rho[i], d_sigma[i], d_dedrho[i], d_dedsigma[i] point to the
 * arrays of system i, d_energy to `count` device doubles.  One launch per
 * stage covers all systems of a part (persistent tile loop); the parts'
 * stage chains are independent branches of one CUDA graph, captured on the
 * first call and replayed (a changed pointer set is uploaded to the
 * descriptors before the replay). */
int vdwgb_batch_calculate_device(vdwgb_batch b, const double *const *d_rho,
                                 const double *const *d_sigma, double *const *d_dedrho,
                                 double *const *d_dedsigma, double *d_energy, void *cuda_stream);
/* The same from HOST arrays: copies in through per-handle device staging,
 * evaluates, copies dedrho, dedsigma and the `count` energies back, and waits.
 * Blocking.  A split batch (see vdwgb_batch_launches) runs each part as its
 * own copy-in / stages / copy-out chain on its own stream, so one part's
 * copies overlap the other parts' kernels; the streams' priorities fall with
 * the part index, so earlier parts finish first and their copies out overlap
 * the later parts' kernels.  Pinned host arrays let the copies run
 * asynchronously (pageable ones work, at the speed of staged copies). */
int vdwgb_batch_calculate(vdwgb_batch b, const double *const *rho, const double *const *sigma,
                          double *const *dedrho, double *const *dedsigma, double *energy);

/* Kernel launches one evaluation of the batch enqueues.  A batch of two or
 * more systems runs as K parts (consecutive systems, split by grid points)
 * whose stage chains are independent branches of the captured graph, so
 * their stages overlap; each part launches its own stages.  K comes from
 * VDWGB_BATCH_SPLIT in the environment when the batch is created (0 or 1:
 * one launch per stage for the whole batch; 2..8; default 6), capped by the
 * number of systems.  Results are the same either way. */
int vdwgb_batch_launches(vdwgb_batch b);

/* Stage timing: with timing enabled, each batch evaluation records CUDA
 * events between its kernel launches (launched directly, not from the
 * graph).  vdwgb_batch_stage_ms waits for the recorded calls, writes the
 * summed milliseconds per stage to ms[vdwgb_num_stages()], the number of
 * calls to *ncalls, and starts a new accumulation. */
int vdwgb_batch_set_timing(vdwgb_batch b, int enable);
int vdwgb_batch_stage_ms(vdwgb_batch b, double *ms, int *ncalls);
int vdwgb_num_stages(void);
const char *vdwgb_stage_name(int i);

int vdwgb_batch_free(vdwgb_batch *b);

/* ---- served form: requests of different grids arriving over time -------- */

typedef struct vdwgb_server_s *vdwgb_server;

typedef struct {
    long long submitted, completed, failed, batches;
    double mean_batch;       /* requests per batched launch */
    double pts_per_s;        /* grid points of completed requests / (last completion - first submit) */
    double p50_s, p99_s;     /* latency quantiles (completion - submission) of completed requests */
    size_t pool_bytes, pool_used_peak;
    long long plans_reused;  /* requests that re-planned a resident plan of their grid */
    long long plans_built;   /* requests that built a new plan */
} vdwgb_server_stats_t;

/* Create a server on `device` for `precision`.  pool_bytes: device-memory
 * budget for admitted requests and resident plans (work buffer, records,
 * k-point order, staging of each); a request is admitted, in arrival order,
 * when a resident plan of its grid is idle, or its footprint fits what is
 * left after evicting idle plans (least recently used first).  A finished
 * request's plan stays resident; the next request of the same grid re-plans
 * only its cell-dependent parts (reciprocal metric, k-point order sorted on
 * the device, chunks).  max_batch (1..256): most requests per batched launch (one launch per
 * stage over all of them); max_inflight (1..8): batches on the GPU at once,
 * each on its own stream, so later requests are admitted and planned while
 * earlier ones run.  At most max_batch (max_inflight + 1) requests are
 * admitted and not yet launched; the rest wait on the host and hold no
 * device memory.  Worker threads plan requests (FFT plans, k-point order),
 * upload inputs with stream-ordered allocations, launch batches and collect
 * results.  The kernel table is built and stays resident. */
int vdwgb_server_new(int device, int precision, size_t pool_bytes, int max_batch, int max_inflight,
                     vdwgb_server *out);

/* Queue one evaluation (grid nx*ny*nz, cell9 = 9 cell doubles as in
 * vdwgb_set_unit_cell).  rho, sigma (read) and dedrho, dedsigma (written)
 * are HOST arrays owned by the caller, valid until the request is reported
 * done.  *id receives the request id.  Never waits for the GPU.  EAGAIN if
 * the request alone exceeds the pool; EINVAL on bad arguments (a grid the
 * planner rejects fails the request, reported by poll/wait). */
int vdwgb_server_submit(vdwgb_server s, int functional, int nx, int ny, int nz, const double *cell9,
                        const double *rho, const double *sigma, double *dedrho, double *dedsigma,
                        long long *id);

/* 1 and energy / latency written if request id is done (the id is then
 * forgotten), 0 if still pending, a negative code if it failed (also
 * forgotten) or is unknown (ENOTFOUND). */
int vdwgb_server_poll(vdwgb_server s, long long id, double *energy, double *latency_s);

/* As poll, but waits up to timeout_s seconds; ETIMEDOUT if still pending. */
int vdwgb_server_wait(vdwgb_server s, long long id, double timeout_s, double *energy, double *latency_s);

int vdwgb_server_stats(vdwgb_server s, vdwgb_server_stats_t *out);

/* Wait (at most 60 s) for batches on the GPU, stop the workers, free
 * everything, set *s = NULL.  Requests not yet reported are dropped. */
int vdwgb_server_free(vdwgb_server *s);

/* ---- slab decomposition over several GPUs ----------------------------------
 * The parallel layout of the paper (Sec. 3, parallelisation: FFTW-MPI slabs
 * over x and the transposed, y-distributed spectrum) as GPU stages of one
 * rank of P.  Rank r owns the real-space x-planes [r nx/P, (r+1) nx/P) (its
 * x-slab: rho, sigma, dedrho, dedsigma as (nx/P) x ny x nz arrays, C order)
 * and the spectrum's y positions [r ny/P, (r+1) ny/P) (its ky-slab).  One
 * evaluation, each call enqueued on cuda_stream:
 *   vdwgb_slab_forward   q0, theta, transforms along z and y on the x-slab
 *   vdwgb_slab_pack      x-slab spectrum -> d_send, ordered by destination rank
 *   (caller) all-to-all of equal parts: d_send of every rank -> d_bspec
 *   vdwgb_slab_contract  transforms along x, kernel contraction and energy on
 *                        the ky-slab, inverse transforms along x; d_energy
 *                        receives this rank's part of E (sum over ranks = E)
 *   (caller) all-to-all back: d_bspec of every rank -> d_recv
 *   vdwgb_slab_unpack    d_recv -> x-slab spectrum
 *   vdwgb_slab_inverse   inverse transforms along y and z and the potential
 *   (caller) sum of the ranks' energies
 * nx and ny must be multiples of P (EINVAL otherwise).  d_aspec and d_bspec
 * (the x-slab and ky-slab work buffers) and the exchange buffers d_send /
 * d_recv are device memory of vdwgb_slab_bytes bytes each, 256-byte aligned,
 * owned by the caller (so the caller's collective library can address them)
 * and kept until vdwgb_slab_free.  Results equal those of one handle on the
 * whole grid: potentials bit for bit, the energy up to the order of its sum.
 * Callers check vdwgb_device_status after synchronising. */
typedef struct vdwgb_slab_s *vdwgb_slab;
size_t vdwgb_slab_bytes(int nx, int ny, int nz, int P, int precision);
int vdwgb_slab_new(int functional, int nx, int ny, int nz, const double *cell9, int P, int rank, int device,
                   int precision, void *d_aspec, void *d_bspec, vdwgb_slab *out);
int vdwgb_slab_forward(vdwgb_slab s, const double *d_rho, const double *d_sigma, void *cuda_stream);
int vdwgb_slab_pack(vdwgb_slab s, void *d_send, void *cuda_stream);
int vdwgb_slab_contract(vdwgb_slab s, double *d_energy, void *cuda_stream);
int vdwgb_slab_unpack(vdwgb_slab s, const void *d_recv, void *cuda_stream);
int vdwgb_slab_inverse(vdwgb_slab s, double *d_dedrho, double *d_dedsigma, void *cuda_stream);
int vdwgb_slab_free(vdwgb_slab *s);

/* ---- allocation-free evaluation ------------------------------------------
 * The paper has no counterpart of this entry point; it serves host codes that
 * must not allocate device memory where they evaluate (a code running inside
 * its own memory pool or budget, or in a region where cudaMalloc is not
 * allowed).  It computes what vdwgb_calculate_device computes for a handle of
 * the same functional and cell in VDWGB_FP32_MIXED precision with cubic
 * interpolation, without a handle and without allocating: every scratch
 * array (work buffer, point records, k-point order, energy partials, plan
 * descriptors) lives in one fixed device array of the library (about
 * 3.4 MiB, held by every GPU that loads the library).
 *
 * Limits: each axis <= 64, nx*ny*nz <= 32768, nx*ny*(nz/2+1) <= 17408, axis
 * lengths with prime factors 2, 3, 5, 7 only; beyond them EINVAL.
 * ESTATE if the device has no resident kernel table yet: call
 * vdwgb_kernel_table(device, NULL, NULL, NULL) once before (that call
 * allocates).  The first call on a device looks up the device address of the
 * fixed array, with the device made current.
 *
 * Arguments: cell9 as in vdwgb_set_unit_cell (host, row-major lattice
 * vectors, Bohr); d_rho, d_sigma (read), d_dedrho, d_dedsigma (written) are
 * DEVICE arrays of nx*ny*nz doubles in C order, d_energy one device double;
 * all enqueued on cuda_stream (NULL = legacy default stream).  The plan data
 * (k-point order, twiddles, descriptors) are copied into the fixed array
 * from pageable host memory, so the call may wait for the stream's earlier
 * work before it returns, and it cannot be captured into a CUDA graph: on a
 * stream that is being captured it returns ESTATE without enqueuing
 * anything.  All calls on one device share its fixed array and leave their
 * data in it (nothing needs clearing: each call overwrites what it reads).
 * Calls on one device whose GPU work overlaps (on two streams, say) race on
 * the array and give wrong results: order them, e.g. on one stream.  Each
 * device has its own array.  A kernel whose bounded wait for staged data ran
 * out sets the device's status flag: after synchronising, check
 * vdwgb_device_status(device) (0: the results are valid). */
int vdwgb_calculate_noalloc(int device, int functional, int nx, int ny, int nz, const double *cell9,
                            const double *d_rho, const double *d_sigma, double *d_dedrho,
                            double *d_dedsigma, double *d_energy, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VDWGB_H */
