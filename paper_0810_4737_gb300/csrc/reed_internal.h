// reed_internal.h -- declarations shared by the host entry points and the
// per-precision kernel translation units.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "reed_common.cuh"

struct LaunchCfg {
    int threads, ctas_per_sm, grid;
    size_t smem;
};

// Per-precision launchers (prec: REED_PREC_MIXED -> float, REED_PREC_FP64 -> double).
namespace reed_f32 {
size_t smem_bytes(int tt, int na, int bond_cap, int adj = 0, int nbins = 0, int act = 0);
size_t spill_bytes(int tt);
size_t adj_scratch_bytes(const DevParams& P, size_t entry);
size_t entry_bytes(int tt, int na);
cudaError_t occupancy(int tt, int threads, size_t smem, int* ctas, int adj = 0);
cudaError_t launch_track(int tt, const DevParams& P, const DevBuf& B, const LaunchCfg& L, cudaStream_t s);
cudaError_t launch_forces(int tt, const DevParams& P, int n, const double* xyz, const int* sp, const double* ion,
                          double* out, unsigned char* spill, size_t smem, cudaStream_t s);
cudaError_t launch_window_replay(const DevParams& P, uint64_t key, const double* path, int npts, int* anchors,
                                 int cap, int* cells, int* bas, double* xyz, int* count, size_t smem,
                                 cudaStream_t s);
cudaError_t launch_cell_atoms(const DevParams& P, uint64_t key, int ix, int iy, int iz, double* xyz, int* sp,
                              int* count, cudaStream_t s);
}  // namespace reed_f32
namespace reed_f64 {
size_t smem_bytes(int tt, int na, int bond_cap, int adj = 0, int nbins = 0, int act = 0);
size_t spill_bytes(int tt);
size_t adj_scratch_bytes(const DevParams& P, size_t entry);
size_t entry_bytes(int tt, int na);
cudaError_t occupancy(int tt, int threads, size_t smem, int* ctas, int adj = 0);
cudaError_t launch_track(int tt, const DevParams& P, const DevBuf& B, const LaunchCfg& L, cudaStream_t s);
cudaError_t launch_forces(int tt, const DevParams& P, int n, const double* xyz, const int* sp, const double* ion,
                          double* out, unsigned char* spill, size_t smem, cudaStream_t s);
cudaError_t launch_window_replay(const DevParams& P, uint64_t key, const double* path, int npts, int* anchors,
                                 int cap, int* cells, int* bas, double* xyz, int* count, size_t smem,
                                 cudaStream_t s);
cudaError_t launch_cell_atoms(const DevParams& P, uint64_t key, int ix, int iy, int iz, double* xyz, int* sp,
                              int* count, cudaStream_t s);
}  // namespace reed_f64
