// Host-side declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "psst_device.cuh"

namespace psst {

// One launch of the CTA/cluster kernel: the networks of one size class.
struct ClassLaunch {
    int cl;               // CTAs per network (1, 2 or 4)
    int n_nets;           // networks in the class
    int block, smem;      // CTA size, dynamic shared memory
    const int *list;      // [n_nets] device: network indices, largest first
    const NetPlan *plans; // [all nets] device
    int lrep_cap;         // per-pair gates: at most 2^lrep_cap copies of the gate table (autotuned)
};

// CTA/cluster batched kernel (psst_cta.cu).
int cta_static_smem();
cudaError_t cta_prepare(int cl, int max_smem);
cudaError_t pair_check(const NetView &v, uint8_t *out, int smem, cudaStream_t stream);
cudaError_t cta_launch(const NetView &v, const ClassLaunch &c, long long step0, int nsteps, cudaStream_t stream);

// Networks without synapses, one thread per neuron (psst_indep.cu).
cudaError_t indep_launch(const NetView &v, const int *ind_neuron, const int *ind_net, int count, long long step0,
                         int nsteps, cudaStream_t stream);

// Grid-wide single-network kernel (psst_grid.cu).
cudaError_t grid_occupancy(int block, int smem, int *blocks_per_sm);
cudaError_t grid_launch(const NetView &v, const GridView &g, long long step0, int nsteps, int grid, int block,
                        int smem, cudaStream_t stream);

// Discrete adjoint (psst_adjoint.cu).
long long adj_smem_need(int N, int nt, int n_items, int K, int n_citems, int KC);
// Floats one step keeps in an adjoint segment buffer (its stages: RK4 four,
// Euler one, a tableau rk_ns).
long long adj_segment_floats(int method, int rk_ns, int N, int nt);
cudaError_t adj_launch(const NetView &v, const AdjView &av, long long step0, int nsteps, int smem, int n_types,
                       float *grad_np, cudaStream_t stream);

}  // namespace psst
