// Device-side control of the captured run: the step counter, the refinement
// and inner-Krylov loop counters and the conditions of the three nested WHILE
// nodes (time steps, refinement passes, inner iterations), so that a whole
// simulation runs as one graph launch without any host round trip.
#include "bt_kernels.cuh"

namespace bt {

// step begin: activity of every system (segments past their echo time stay
// frozen), the count of live systems, and the refinement pass counter
__global__ void k_graph_step_begin(GraphCtl c, int* rf_active) {
  const int step = c.ctl[0];
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < c.G * c.R; s += blockDim.x) {
    const int a = step <= c.segN[s / c.R] ? 1 : 0;
    rf_active[s] = a;
    if (a) atomicAdd(&live, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c.n_active[1] = live;
    c.ctl[1] = 0;
  }
}

// which = 0: before the refinement loop (condition: live systems)
//         1: end of a refinement pass (live systems and passes left)
//         2: before the inner loop (condition: active systems)
//         3: end of an inner iteration (active systems and iterations left)
//         4: before the first and after every time step (steps left)
__global__ void k_graph_cond(GraphCtl c, int which, cudaGraphConditionalHandle h) {
  unsigned int v = 0;
  if (which == 4) {
    v = c.ctl[0] <= c.n_steps;
  } else if (which == 0) {
    v = c.n_active[1] > 0;
  } else if (which == 1) {
    const int p = ++c.ctl[1];
    ++c.ctl[4];
    v = c.n_active[1] > 0 && p < c.max_refine;
  } else if (which == 2) {
    c.ctl[2] = 0;
    v = c.n_active[0] > 0;
  } else {
    const int it = ++c.ctl[2];
    ++c.ctl[3];
    v = c.n_active[0] > 0 && it < c.max_iter;
  }
  cudaGraphSetConditional(h, v);
}

__global__ void k_graph_step_end(GraphCtl c) { ++c.ctl[0]; }

void launch_graph_step_begin(const GraphCtl& c, int* rf_active, cudaStream_t st) {
  k_graph_step_begin<<<1, 256, 0, st>>>(c, rf_active);
}
void launch_graph_cond(const GraphCtl& c, int which, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_graph_cond<<<1, 1, 0, st>>>(c, which, h);
}
void launch_graph_step_end(const GraphCtl& c, cudaStream_t st) { k_graph_step_end<<<1, 1, 0, st>>>(c); }

}  // namespace bt
