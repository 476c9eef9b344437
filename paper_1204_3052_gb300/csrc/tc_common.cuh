// Parameter blocks shared by the tensor-core product kernels.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace mp {

struct TcProblem {
  CUtensorMap ax[3];  // X as the A operand: its planes (box 64 x 128)
  CUtensorMap by[3];  // Y as the B operand: its planes (box 64 x 64)
  CUtensorMap cx[3];  // C's planes as TMA store targets (box 64 x 128)
  GemmDesc d;
};

// Up to two products of one level, passed by value (__grid_constant__).
struct TcPairParams {
  TcProblem p[2];
  int count;
  int tiles0;  // tiles of the first product
};

}  // namespace mp
