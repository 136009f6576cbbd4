// sp_kernels.h -- host-callable launchers of the kernels in sp_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "sp_device.cuh"

namespace sp {

cudaError_t launch_reset(const RegionArgs &a, cudaStream_t st);
// 16 cost-model features per region of the launch into X [total][16].
cudaError_t launch_features(const RegionArgs &a, const float4 *simf, const unsigned long long *prev_trace, float *X,
                            cudaStream_t st);
size_t region_smem_bytes(int max_B, int n_tabs, int n_sims, int imp_units);
cudaError_t region_occupancy(int threads, int B, size_t smem, int *blocks_per_sm);
cudaError_t launch_region(const RegionArgs &a, int threads, int max_B, size_t smem, int grid, cudaStream_t st);
cudaError_t launch_sweep(const float2 *phi_in, float2 *phi_out, float4 *pc, const int n[3],
                         const LevelCoef *coef, int lvl, PhysConst q, cudaStream_t st);
int energy_blocks(const int n[3]);
cudaError_t launch_energy(const float2 *phi, const float4 *pc, const int n[3], double inv_dx2, double eta2,
                          double half_lambda_a2, double *partial, double *out, cudaStream_t st);
cudaError_t launch_winding(const float2 *phi, const int n[3], signed char *w, unsigned long long *counts,
                           cudaStream_t st);

}  // namespace sp

namespace sp {
// The base-32 cluster kernel (sp_octant.cu): shared memory per CTA, the
// number of 8-CTA clusters that fit the device, its launch and worker count.
size_t region_oct_smem_bytes(int imp_units, int face_units);
cudaError_t region_oct_clusters(size_t smem, int *clusters);
cudaError_t launch_region_oct(const RegionArgs &a, size_t smem, int clusters, cudaStream_t st);
int region_oct_workers();
}  // namespace sp

namespace sp {
// The 4-cube lattice kernel (sp_lattice.cu): dynamic shared memory of one
// region, worker counts, occupancy, the per-call reset (ticket counter,
// error word, layer epoch) and the launch.
size_t lattice_smem_bytes(int n_slots, int n_foot, int rb_side, int max_cell_n);
bool lattice_valid_threads(int threads);
cudaError_t lattice_occupancy(int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_lattice_reset(Ctl *ctl, int layers, cudaStream_t st);
cudaError_t launch_lattice(const LatArgs &a, int threads, size_t smem, int grid, cudaStream_t st);
}  // namespace sp
