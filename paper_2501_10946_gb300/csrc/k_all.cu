// The kernels of the force step compiled as one translation unit, so that the persistent
// batched step (k_persist.cuh) calls the per-block bodies of every kernel directly.
#include "k_cells.cu"
#include "k_sample.cu"
#include "k_near.cu"
#include "k_forces.cu"
#include "k_persist.cuh"
