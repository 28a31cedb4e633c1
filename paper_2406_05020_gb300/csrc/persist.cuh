// Persistent execution of a phased plan (see persist.cu).
#pragma once
#include "common.cuh"

namespace gpfvm {

class Plan;
struct PersistProg;

// Builds the persistent form of a finalized plan: every phase (the merged
// launch units and typed TC / SCALE / COPY ops of one zip level, or one
// unphased GEMM / GEMV / typed op) becomes a list of work items.  Returns
// null when the plan holds a host callback (FUNC op) or is empty.
// `sync` points at two zeroed device words used by the grid barrier, and
// `status` receives DEV_TIMEOUT if a barrier or tensor-core wait gives up.
PersistProg* persist_build(const Plan& plan, unsigned int* sync, int* status);
void persist_free(PersistProg* prog);
// One cooperative launch of the plan on st.  Returns false (nothing
// launched) if the device cannot hold the grid; the caller then runs the
// plan launch by launch.
bool persist_run(const PersistProg* prog, cudaStream_t st);
// True when GPFVM_PERSIST=1 selects persistent execution of the iteration plans.
bool persist_enabled();

}  // namespace gpfvm
