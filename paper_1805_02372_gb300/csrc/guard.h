// No exception crosses the C interface: an entry point runs the calls that may throw
// (C++ containers growing on the host) through guarded(), which turns a failed host
// allocation (std::bad_alloc, or std::length_error for a size no container can hold)
// into PA_ERR_NOMEM and any other exception into PA_ERR_INVALID.
#pragma once

#include <new>
#include <stdexcept>

#include "../../include/pa.h"

namespace pa {

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
