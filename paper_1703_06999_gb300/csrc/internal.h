// Internal interfaces shared by the C ABI (capi.cu) and the serving loop
// (serve.cu).  Not part of the public header.
#pragma once
#include <cstddef>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/vdwgb.h"
#include "common.cuh"
#include "pipeline.h"
#include "table.h"

struct vdwgb_data {
    int functional = 1;
    int interp = VDWGB_INTERP_CUBIC;
    int nx = 0, ny = 0, nz = 0;
    double cell[9] = {0};
    bool cell_set = false;
    bool inited = false;
    int device = -1;
    int prec = VDWGB_FP64;
    // device memory
    void *spec = nullptr;
    bool spec_external = false;        // spec belongs to the caller (slab decomposition)
    void *rec = nullptr;
    double *epart = nullptr;
    void *tw[3] = {nullptr, nullptr, nullptr};
    unsigned *kidx = nullptr;
    int4 *chunks = nullptr;
    unsigned short *kord = nullptr;    // plane kernel k-point order
    void *tmap = nullptr;              // FP32: tensor maps of the x / y pass tiles
    int nbatch = 0;                    // live batches built on this handle (they share tmap)
    vdwgb::SysDev *dsys = nullptr;
    int *dprefix = nullptr;
    vdwgb::SysDev hsys;
    vdwgb::LaunchSet ls;
    const void *table = nullptr;
    size_t bytes = 0;
    // host-pointer path staging
    double *d_io = nullptr;      // n, sigma, dedn, dedsigma, energy
    // spin-polarised form (spin.cu), allocated at its first call: n and q0
    // (overwritten by the two potential sums), four derivatives of q0; host
    // path staging of four inputs, four outputs and the energy
    double *d_spin = nullptr;
    double *d_spin_io = nullptr;
    // a caller's kernel table (vdwgb_set_kernel_k): its k-space values, and
    // the spline coefficients built from them at init (the resident table
    // otherwise)
    std::vector<double> kernel_k;
    vdwgb::CustomTable ktab;
    cudaStream_t stream = nullptr;
    cudaStream_t alloc_stream = nullptr;   // set: stream-ordered allocations (server handles)
    const double *last_ptr[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace vdwgb {

int fail(int code, const char *fmt, ...);
// cudaMalloc, failing with cudaErrorMemoryAllocation while an allocation
// fault is injected (vdwgb_inject_fault)
cudaError_t device_malloc(void **p, size_t bytes);
int cuda_fail(cudaError_t e, const char *what);
int device_setup(int device);
bool device_peek(int device, int *sms, size_t *maxsmem, int **err);
// plan and allocate a handle (cell already set); alloc_stream != 0 makes
// every allocation and upload stream-ordered on it
int handle_init(vdwgb_data *h, int device, int precision, cudaStream_t alloc_stream);
void handle_release(vdwgb_data *h);
// re-plan an initialised handle for another cell and functional of the same
// grid and precision: metric, k-point order and chunks (on the device),
// descriptor; buffers, twiddles, tiles and tensor maps are kept.  Waits for
// the handle's stream (alloc_stream for server handles).
int handle_replan(vdwgb_data *h, const double *cell9, int functional);
// pieces of a plan for the slab decomposition (slab.cu): I/O pointers of the
// descriptor (uploaded on st if changed), the k-point order and chunks of the
// current descriptor (device sort; waits for st), the descriptor, prefix sums
// and tensor maps, a caller-owned work buffer in place of the handle's own
int handle_set_io(vdwgb_data *h, const double *n, const double *s, double *dn, double *ds, double *e,
                  cudaStream_t st);
int handle_sort_kpoints(vdwgb_data *h, cudaStream_t st);
int handle_upload_plan(vdwgb_data *h);
void handle_use_spec(vdwgb_data *h, void *spec);
int device_sms(int device);
size_t handle_io_bytes(const vdwgb_data *h);
// launch set over n handles: fills hdesc[n] (copies of the handles'
// descriptors; the caller sets I/O pointers), hprefix[NKIND * (n + 1)] and L,
// whose device pointers are ddesc / dprefix (filled by the caller's copy)
int batch_launchset(vdwgb_data *const *hs, int n, SysDev *hdesc, int *hprefix, const SysDev *ddesc,
                    const int *dprefix, LaunchSet &L);

}  // namespace vdwgb
