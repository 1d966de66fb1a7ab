// Mixed-precision solvers with FP64 iterative refinement (placeholder until
// the kernels land; reports no configurations so the API rejects the modes).
#include "ss_internal.h"

namespace ss {
int mixed_config_count(int, int) { return 0; }
const Config *mixed_config_get(int, int, int) { return nullptr; }
long long mixed_scratch_per_n2(int, int) { return 0; }
cudaError_t launch_mixed(int, const Operands &, const Sched &, const Launch &, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace ss
