// Resident kernel table (table.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace vdwgb {

struct TableRefs {
    const double *phir;     // [NPAIR][NR + 1]
    const double *phik;     // [NPAIR][NK]
    const dvec4 *cub64;   // [NK - 1][NPAIR] interval polynomials, cubic spline
    const dvec4 *lin64;   // linear interpolation
    const float4 *cub32;
    const float4 *lin32;
    double seconds;
};

// Build (once per device and process) and return the resident table.
cudaError_t table_get(int device, TableRefs &out);
double table_seconds(int device);
bool table_peek(int device, TableRefs &out);
cudaError_t table_phi(int device, int npts, const double *d1, const double *d2, double *out);
void host_qmesh(QMeshDev &q);

// A caller's kernel table: spline coefficients built like the resident
// table's from its k-space values (NPAIR x NK FP64, host), on the current
// device; freed with table_custom_free.
struct CustomTable {
    dvec4 *cub64 = nullptr, *lin64 = nullptr;
    float4 *cub32 = nullptr, *lin32 = nullptr;
};
cudaError_t table_custom(const double *h_phik, CustomTable &out, cudaStream_t st);
void table_custom_free(CustomTable &t);

}  // namespace vdwgb
