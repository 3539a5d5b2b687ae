// shapes.h -- the CTA / cluster shapes of the evolution kernel that the library is built with,
// and their launch.  A shape is (P grid nodes per thread, NT threads per CTA, CL CTAs per
// instance); one instance of N points fits a shape when the CL CTAs hold its N - 1 cells
// (P * NT * CL >= N - 1) and every CTA gets at least one block of P nodes.
#pragma once

#include <cuda_runtime.h>

#include "evolve.cuh"

namespace adscl {

struct Shape {
    int P, NT, CL;
};

constexpr int kNumShapes = 18;
extern const Shape kShapes[kNumShapes];

// index of the shape (P, NT, CL) in kShapes, or -1
int shape_index(int P, int NT, int CL);

// the shape fits grid size N
bool shape_fits(int id, int N);

// padded shared-memory field length and dynamic shared memory of shape id for grids up to Nmax
int shape_stride(int id, int Nmax);
size_t shape_smem(int id, int Nmax);

// raise the dynamic shared-memory limit of every shape's kernel to what it can need
cudaError_t shapes_set_attributes();

// co-resident units (CTAs for CL = 1, clusters otherwise) of shape id on the device with the
// given dynamic shared memory
cudaError_t shape_max_units(int id, size_t smem, int num_sms, int *units);

// launch `units` persistent units of shape id
cudaError_t shape_launch(int id, const EvolveArgs &a, int units, size_t smem, int stride,
                         cudaStream_t stream);

}  // namespace adscl
