// Host interface of the persistent stage kernel (ens_persist.cu).
#pragma once

#include "ens_internal.h"

#include <vector>

namespace ens {

// work-item kinds, in the order of an RK stage's passes
enum : int { kPIX = 0, kPIY, kPZ, kPFY, kPFX, kPFIN, kPKinds };
constexpr int kPSlots = 3;   // grid-size groups one launch can hold (128, 256, 384)

// One work item: `count` consecutive column tiles from tile `a` of field `b`
// (IX, IY, FY, FX), `count` z-pass row groups from row group `a` (Z), or the
// stage finish (FIN), of member m (index in its group) of group `slot`.
struct PItem {
    int kind, slot, m, a, b, count;
};

struct PStageArgs {
    Geo g[kPSlots];
    MemberDev *md;
    const PItem *items;
    int nitems;
    unsigned *next;   // item counter, zero at launch
    unsigned *abort;  // set once a dependency wait gave up, zero at launch
    unsigned *done;   // [global member][kPKinds] items done, zero at launch
    unsigned need[kPSlots][kPKinds];   // items of each kind per member
    int stage, last;
};

bool persist_size_supported(int N);
void persist_items(const std::vector<Geo> &groups, std::vector<PItem> &items, unsigned need[kPSlots][kPKinds]);
cudaError_t persist_prepare();
int persist_ctas_per_sm();
cudaError_t launch_stage_persist(const PStageArgs &a, int ctas, cudaStream_t s);

}  // namespace ens
