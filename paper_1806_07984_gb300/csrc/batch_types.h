// Host/device data of the batched step (see batch.cuh).
#pragma once
#include <cstdint>

#include "basis.h"

namespace ader {

struct BatchInstance {
  int32_t order;    // N
  int32_t side;     // cells per direction (periodic unit square / cube)
  int64_t ncells;   // side^dim
  int64_t u_off;    // offset (doubles) of this instance in u / ustar
  int64_t f_off;    // offset (doubles) of this instance in the face arrays
  double inv_h;     // side / L
  double cfl;       // dt = cfl / max sum_d lambda_d / h_d
};

struct BatchItem {
  int32_t inst;
  int32_t first;   // first cell (or face) of the tile
  int32_t count;   // cells (or faces) in the tile
  int32_t pad;
};

struct BatchArgs {
  const BatchInstance* inst;
  int32_t ninst;
  const BatchItem* items;   // cell tiles (predictor, corrector)
  int32_t nitems;
  const BatchItem* fitems;  // face tiles (Riemann)
  int32_t nfitems;
  double* u;
  double* ustar;
  double* faceQ;
  double* faceF;
  double* fstar;
  double* dt;                // per instance
  unsigned long long* rate;  // per instance, FP64 bits
  int32_t* counters;         // work queues, one per phase launch
  const BasisTables* B;      // indexed by order
  double gamma;
  int32_t iters;             // Picard iterations; 0 selects order + 1
  uint32_t* status;
};

}  // namespace ader
