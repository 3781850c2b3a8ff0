// Device table builder interface (see tables.cu).
#pragma once

#include "common.cuh"

namespace celer {

struct MaterialData {
  double ne;      // electrons / cm3
  double Z, X0, I;
  double f_pe;    // photoelectric scale relative to water
  double f_pair;  // pair-production scale relative to water
};

struct TableBuild {
  int n_mat;
  const MaterialData* mats;  // device array
  int processes;
  double cut_moller, cut_brems;
  double lnEmin, dl;
};

// Fill d_tables ([mat][kCols][kGrid] double2) on the stream; d_scratch holds
// table_scratch_doubles(n_mat) doubles.
cudaError_t build_tables(const TableBuild& tb, double2* d_tables, double* d_scratch, cudaStream_t stream);
size_t table_scratch_doubles(int n_mat);

}  // namespace celer
