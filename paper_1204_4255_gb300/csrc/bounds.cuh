// bounds.cuh -- index checks of the bounds-checking build (-DXSDE_BOUNDS=1).
//
// In that build every global-memory index a kernel computes for a field, a
// table, a sampling buffer or a bulk / tensor copy is checked against the
// extent of its buffer before the access: an index outside records ST_BOUNDS
// in the problem's device status word (xsde_synchronize reports it as
// XSDE_EBOUNDS) and the access is skipped.  In the default build the checks
// compile away.
#pragma once

#include <cstdint>

#ifndef XSDE_BOUNDS
#define XSDE_BOUNDS 0
#endif

namespace xsde {

enum { ST_BOUNDS = 8 };

__device__ __forceinline__ bool bounds_ok(int64_t i, int64_t n, int *status) {
#if XSDE_BOUNDS
    if (i < 0 || i >= n) {
        if (status) atomicOr(status, ST_BOUNDS);
        return false;
    }
#endif
    return true;
}

}  // namespace xsde

// true when 0 <= i < n (always true without XSDE_BOUNDS)
#define XSDE_IN(i, n, status) ::xsde::bounds_ok((int64_t)(i), (int64_t)(n), (status))
