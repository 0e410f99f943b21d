// Device status bits OR-ed into a context's status word by the kernels.
#pragma once
#include "../../include/pmd.h"
namespace pmd {
enum : int {
    ST_NEIGH = 1,
    ST_NONFINITE = 2,
    ST_TIMEOUT = 4,
    ST_LOSTATOM = 8,
    ST_BADNEIGH = 16,   // a neighbour list was found asymmetric (internal invariant)
    ST_BADARG = 32,     // a device-side argument was invalid
};
}  // namespace pmd
