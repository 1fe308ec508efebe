// ivb_compile.h -- host tape validation and compilation into the device
// program format of ivb_internal.h (implemented in ivb_compile.cpp).
#pragma once
#include <string>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_internal.h"

namespace ivb {

// "" for a valid tape, else the reason it is rejected (ivb_create_problem's IVB_ETAPE cases)
std::string validate_tape(const ivb_tape* t);

// point / tangent sweep, per-output adjoint programs, constants, frame layout
// and operation counts of a validated tape; "" on success
std::string compile_tape(const ivb_tape* t, HostProgram& P, std::vector<Ins>& ins, std::vector<RIns>& rins,
                         std::vector<double>& consts);

}  // namespace ivb
