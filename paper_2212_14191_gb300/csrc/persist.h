// Internal interface of the persistent batch engine (persist.cu), used by the batch plan of
// batch.cu for the operations at N >= 2^14.
#pragma once
#include <vector>

#include "common.cuh"

namespace fhe {

struct PersistPlan;

// Plans the operations ops[idx[k]] (NTT, INTT and HMULT at N >= 2^14, validated by the caller):
// tile order, dependency counters and the scratch layout, with at most `slot_budget` bytes of
// HMULT scratch slots (at least one slot). Allocates the plan's device tables.
int persist_create(const fhe_ctx* ctx, const fhe_op* ops, int n, const std::vector<int>& idx, size_t slot_budget,
                   PersistPlan** out);
size_t persist_scratch_bytes(const PersistPlan* p);
size_t persist_tiles(const PersistPlan* p);
// Enqueues one run on `st`: a reset of the counters and one persistent launch. The first run on
// a scratch buffer (and the first after a change of buffer) uploads the tables, which hold
// absolute addresses inside it, synchronously; it must not happen during stream capture.
int persist_run(PersistPlan* p, void* scratch, cudaStream_t st);
void persist_destroy(PersistPlan* p);
// Runs the persistent kernel on one tile whose dependency can never be met, with the given
// wait limit: the wait expires, FHE_ETIMEOUT is recorded in the context's status word and the
// kernel finishes.
int persist_selftest_timeout(const fhe_ctx* ctx, long long limit_cycles, cudaStream_t st);

}  // namespace fhe
