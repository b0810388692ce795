// Integration (RK4, Euler or a tableau) of networks without synapses:
// every neuron is an independent ODE system (the uncoupled systems of the
// paper's Fig. 2b benchmark), so no stage needs a barrier.  One thread owns one neuron for
// all steps of a launch, with its state, its RK4 sums and its parameters in
// registers; the right-hand side and the stage updates are the functions
// the coupled kernels use (psst_syn.cuh), called with a zero synaptic
// current, so results are bitwise those of the coupled kernels for the same
// neurons.
#include <cuda_runtime.h>

#include "psst_device.cuh"
#include "psst_internal.h"
#include "psst_syn.cuh"

namespace psst {

namespace {

constexpr int INDEP_THREADS = 256;

// One stage of kind ST (psst_syn.cuh) of one neuron; ysc/ysn are this and
// the next stage's gates.
template <int ST>
__device__ __forceinline__ float indep_stage(const NetView &v, float V, const float *ysc, float *ysn, float *y0,
                                             float *ylo, float *acc, const float *prm, float iext, float dt) {
    const StageCT<ST> sg{stage_coef<ST>(v, dt)};
    neuron_gates(sg, 0, 1, V, ysc, ysn, y0, ylo, acc);
    return neuron_v(sg, 0, 1, V, ysc, y0, ylo, acc, prm, iext, 0.0f);
}

// Thread t integrates neuron ind_neuron[t] of network ind_net[t] for nsteps
// steps from global step step0 (kernel arguments ordered like net_kernel's
// so that CUDA-graph replay patches step0 at the same position).
__global__ void __launch_bounds__(INDEP_THREADS) indep_kernel(NetView v, const int *ind_neuron, const int *ind_net,
                                                              long long step0, int nsteps, int count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long gi = ind_neuron[t];
    const int b = ind_net[t];
    float y0[4], ylo[4], acc[4], ysa[3], ysb[3], prm[PSST_NEURON_NPARAM];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        y0[x] = v.state[(long long)x * v.N + gi];
        ylo[x] = v.state_lo ? v.state_lo[(long long)x * v.N + gi] : 0.0f;
        acc[x] = 0.0f;
        if (x > 0) ysa[x - 1] = y0[x];
    }
    const float *p = v.nparams + (long long)v.neuron_type[gi] * PSST_NEURON_NPARAM;
    prm[NP_C] = 1.0f / p[NP_C];
#pragma unroll
    for (int x = 1; x < PSST_NEURON_NPARAM; ++x) prm[x] = p[x];
    const float i_const = v.i_const[gi], pulse = v.pulse_amp ? v.pulse_amp[gi] : 0.0f;
    const long long pon = v.pulse_on[b], poff = v.pulse_off[b];
    const float dt = v.dt;
    float V = y0[0];
    int rec_phase = v.rec_stride > 0 ? (int)((step0 + 1) % v.rec_stride) : -1;
    for (int itn = 0; itn < nsteps; ++itn) {
        const long long step = step0 + itn;
        const float iext = input_current(v, i_const, pulse, step >= pon && step < poff, gi, step);
        if (v.method == PSST_METHOD_EULER) {
            // one stage per step; the gates alternate between ysa and ysb by step
            if (itn & 1) V = indep_stage<4>(v, V, ysb, ysa, y0, ylo, acc, prm, iext, dt);
            else V = indep_stage<4>(v, V, ysa, ysb, y0, ylo, acc, prm, iext, dt);
        } else if (v.method == PSST_METHOD_TABLEAU) {
            // stage s of step itn reads the gates of parity (itn * n + s) & 1
#define PSST_TAB_STAGE(n, s)                                                                                    \
    V = (((itn * (n) + (s)) & 1) ? indep_stage<tableau_stage(n, s)>(v, V, ysb, ysa, y0, ylo, acc, prm, iext, dt)         \
                                 : indep_stage<tableau_stage(n, s)>(v, V, ysa, ysb, y0, ylo, acc, prm, iext, dt))
            switch (v.rk_ns) {
            case 1: PSST_TAB_STAGE(1, 0); break;
            case 2: PSST_TAB_STAGE(2, 0); PSST_TAB_STAGE(2, 1); break;
            case 3: PSST_TAB_STAGE(3, 0); PSST_TAB_STAGE(3, 1); PSST_TAB_STAGE(3, 2); break;
            default: PSST_TAB_STAGE(4, 0); PSST_TAB_STAGE(4, 1); PSST_TAB_STAGE(4, 2); PSST_TAB_STAGE(4, 3); break;
            }
#undef PSST_TAB_STAGE
        } else {
            // stage gates alternate between ysa (even stages read) and ysb
            V = indep_stage<0>(v, V, ysa, ysb, y0, ylo, acc, prm, iext, dt);
            V = indep_stage<1>(v, V, ysb, ysa, y0, ylo, acc, prm, iext, dt);
            V = indep_stage<2>(v, V, ysa, ysb, y0, ylo, acc, prm, iext, dt);
            V = indep_stage<3>(v, V, ysb, ysa, y0, ylo, acc, prm, iext, dt);
        }
        if (rec_phase >= 0) {
            if (rec_phase == 0) v.rec[(((step + 1) / v.rec_stride - 1) % v.rec_cap) * v.N + gi] = V;
            rec_phase = rec_phase + 1 == v.rec_stride ? 0 : rec_phase + 1;
        }
    }
    bool bad = false;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        bad |= !isfinite(y0[x]);
        v.state[(long long)x * v.N + gi] = y0[x];
        if (v.state_lo) v.state_lo[(long long)x * v.N + gi] = ylo[x];
    }
    if (bad) set_error(v.err, PSST_ERR_NONFINITE);
}

}  // namespace

cudaError_t indep_launch(const NetView &v, const int *ind_neuron, const int *ind_net, int count, long long step0,
                         int nsteps, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    const int grid = (count + INDEP_THREADS - 1) / INDEP_THREADS;
    indep_kernel<<<grid, INDEP_THREADS, 0, stream>>>(v, ind_neuron, ind_net, step0, nsteps, count);
    return cudaGetLastError();
}

}  // namespace psst
