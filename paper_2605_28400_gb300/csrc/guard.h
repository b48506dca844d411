// guard.h — the C ABI's no-throw rule. Every entry point returns a trioseq_status and never lets a
// C++ exception cross the C boundary: host allocation failures (std::bad_alloc, and
// std::length_error from an impossible container size) become TRIOSEQ_ENOMEM, anything else
// TRIOSEQ_EINVAL. The library itself throws nothing; exceptions come only from the standard
// containers and threads it uses.
//
// Host fault injection for tests: with TRIOSEQ_TEST_HOST_BAD_ALLOC set to a non-zero value in the
// environment when the first guarded call runs, every guarded call fails as if its first host
// allocation had thrown, before it touches its arguments or the GPU.
#pragma once
#include <cstdlib>
#include <new>
#include <stdexcept>

#include "trioseq.h"

namespace trioseq {

inline bool host_bad_alloc_injected() {
  static const bool on = [] {
    const char* v = std::getenv("TRIOSEQ_TEST_HOST_BAD_ALLOC");
    return v && *v && !(v[0] == '0' && v[1] == 0);
  }();
  return on;
}

template <class F>
trioseq_status no_throw(F&& f) noexcept {
  try {
    if (host_bad_alloc_injected()) throw std::bad_alloc();
    return f();
  } catch (const std::bad_alloc&) {
    return TRIOSEQ_ENOMEM;
  } catch (const std::length_error&) {
    return TRIOSEQ_ENOMEM;
  } catch (...) {
    return TRIOSEQ_EINVAL;
  }
}

}  // namespace trioseq
