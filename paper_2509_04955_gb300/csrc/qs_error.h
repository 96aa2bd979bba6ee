// Error type thrown by the host runtime and mapped to qs_status at the C ABI.
#pragma once
#include <stdexcept>
#include <string>

#include "qsim_gb300.h"

namespace qs {
struct Error : std::runtime_error {
  qs_status code;
  Error(qs_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
}  // namespace qs
