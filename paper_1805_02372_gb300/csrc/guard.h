// Rules shared by the entry points of the C interface.
//
// Sizes: no key or output longer than kMaxBits is accepted (the seed index n+m-2 must fit
// comfortably); sizes_valid() is checked before anything else runs, the autotuner's
// calibration included.
//
// No exception crosses the interface: an entry point runs the calls that may throw
// (C++ containers growing on the host) through guarded(), which turns a failed host
// allocation (std::bad_alloc, or std::length_error for a size no container can hold)
// into PA_ERR_NOMEM and any other exception into PA_ERR_INVALID.
#pragma once

#include <stdint.h>

#include <new>
#include <stdexcept>

#include "../../include/pa.h"

namespace pa {

constexpr uint64_t kMaxBits = uint64_t(1) << 40;

inline bool sizes_valid(uint64_t n, uint64_t m) {
    return n != 0 && m != 0 && n <= kMaxBits && m <= kMaxBits;
}

template <class F>
int guarded(F &&body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return PA_ERR_NOMEM;
    } catch (const std::length_error &) {
        return PA_ERR_NOMEM;
    } catch (...) {
        return PA_ERR_INVALID;
    }
}

}  // namespace pa
