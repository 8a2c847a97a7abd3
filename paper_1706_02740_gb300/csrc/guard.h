// No C++ exception leaves the library: entry points whose work allocates host memory or starts
// threads run their body through guarded(), which turns std::bad_alloc into SFT_ENOMEM and any
// other standard exception into SFT_EINVAL, with the message in sft_last_error().
#pragma once

#include <exception>
#include <new>
#include <string>

#include "sft_internal.h"

namespace sft {

template <typename F>
sft_status guarded(const char* who, F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    set_error(std::string(who) + ": host allocation failed");
    return SFT_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string(who) + ": " + e.what());
    return SFT_EINVAL;
  } catch (...) {
    set_error(std::string(who) + ": unexpected failure");
    return SFT_EINVAL;
  }
}

}  // namespace sft
