// Thread-block admission of the serving loop (host code only, no CUDA).
//
// Every request is solved by one cooperative grid whose blocks must all be
// resident at the same time (they wait for each other at grid barriers).
// Grids of different requests run side by side, so the server admits a
// request only when its blocks are sure to find room next to the blocks of
// the requests already running, whatever SMs the hardware put those on.
//
// Requests come in two classes, fixed before admission together with the
// launch shape that the solve will use:
//   SMALL - 256-thread blocks of which `small_per_sm` fit on one SM;
//   FULL  - blocks that take a whole SM (512-thread blocks compiled for one
//           block per SM, possibly with the shared-memory operator).
// Invariants kept by can_admit (sms = SM count):
//   full_in_use + small_in_use <= sms          (before admitting a FULL grid:
//       every SMALL block may sit on an SM of its own, and a FULL grid needs
//       that many SMs with nothing else on them)
//   small_in_use <= small_per_sm * (sms - full_in_use)   (SMALL blocks fit on
//       the SMs that no FULL block holds)
// Both hold after every admission, so every admitted grid is co-resident.
#pragma once
#include <stdint.h>
#include <algorithm>

namespace nnqp {

enum AdmitClass { ADMIT_SMALL = 0, ADMIT_FULL = 1 };

struct RequestShape {
    int cls = ADMIT_SMALL;
    int tpb = 256;       // threads per block of the solve launch
    int blocks = 1;      // blocks of the solve launch
};

// Launch shape of a request whose reduced system has at most `slices`
// 32-row slices (the server knows only the node count before assembly, an
// upper bound of the free unknowns).  It follows the single-system sizing:
//   - systems of at most 4 * sms / 2 slices: 256-thread blocks, one block per
//     8 slices (SMALL);
//   - mid-size systems (up to 32 slices per SM): one 512-thread block per SM
//     at most, one per 8 slices (FULL);
//   - larger systems: the whole co-resident grid of 256-thread blocks
//     (SMALL, every unit: the request runs alone).
// share > 0 caps the blocks of one request (sm_share_blocks).
inline RequestShape request_shape(int64_t slices, int sms, int small_per_sm, int share) {
    RequestShape r;
    const int64_t cap_small = (int64_t)small_per_sm * sms;
    const int64_t by8 = std::max<int64_t>(1, (slices + 7) / 8);
    if (slices > (int64_t)8 * sms / 2 && slices <= (int64_t)32 * sms) {
        r.cls = ADMIT_FULL;
        r.tpb = 512;
        r.blocks = (int)std::min<int64_t>(by8, sms);
    } else if (slices > (int64_t)32 * sms) {
        r.cls = ADMIT_SMALL;
        r.tpb = 256;
        r.blocks = (int)cap_small;
    } else {
        r.cls = ADMIT_SMALL;
        r.tpb = 256;
        r.blocks = (int)std::min<int64_t>(by8, cap_small);
    }
    if (share > 0) r.blocks = std::max(1, std::min(r.blocks, share));
    return r;
}

// Blocks of the running grids, by class.
struct BlockLedger {
    int sms = 1, small_per_sm = 1;
    int full_in_use = 0, small_in_use = 0;

    bool can_admit(const RequestShape &r) const {
        if (r.cls == ADMIT_FULL) return full_in_use + r.blocks + small_in_use <= sms;
        return (int64_t)small_in_use + r.blocks <= (int64_t)small_per_sm * (sms - full_in_use);
    }
    // A request that cannot run even on an idle device (never admitted).
    bool fits_alone(const RequestShape &r) const {
        return r.cls == ADMIT_FULL ? r.blocks <= sms : r.blocks <= small_per_sm * sms;
    }
    void admit(const RequestShape &r) { (r.cls == ADMIT_FULL ? full_in_use : small_in_use) += r.blocks; }
    void release(const RequestShape &r) { (r.cls == ADMIT_FULL ? full_in_use : small_in_use) -= r.blocks; }
};

}  // namespace nnqp
