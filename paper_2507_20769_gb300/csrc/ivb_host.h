// ivb_host.h -- host-side interval evaluation of a tape for the branch and
// bound around the GPU bounding kernels: point upper bounds, the descent
// corner heuristic and forward-backward constraint propagation (bound
// tightening of node boxes before they are bounded). Outward rounding on
// the CPU; same value, tangent and adjoint rules as the kernels.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/ivb.h"

namespace ivb {

struct HostTape {
    int n = 0, T = 0, no = 0, obj = 0;
    bool has_eq = false;
    std::vector<ivb_op> ops;
    std::vector<int32_t> out_idx;
    std::vector<uint8_t> out_kind;
};

struct hiv {
    double lo, hi;
};

// copy of a validated tape
void host_tape(const ivb_tape* t, HostTape& H);

// interval value of every entry on the box ([n][2] lo, hi)
void host_values(const HostTape& H, const double* box, hiv* V);

// enclosure of the gradient of output o over the box, forward tangents
// (grad_mode IVB_GRAD_FORWARD) or the reverse adjoint sweep; G[n]
void host_gradient(const HostTape& H, const double* box, int o, int grad_mode, hiv* G);

// hi(f([x,x])) when every inequality has hi(g([x,x])) <= 0 and there are no
// equalities, else +inf: a rigorous upper bound on the constrained minimum
double host_point_value(const HostTape& H, const double* x);

// descent corner of the box (per dimension: lo where the objective's
// gradient enclosure is > 0, hi where < 0, the centre otherwise), else the
// midpoint between that corner and the centre: host_point_value there
double host_corner_value(const HostTape& H, const double* box, int grad_mode);

// Forward-backward bound tightening (HC4-style projections): the interval
// value of every entry on the box, intersected with [-inf, 0] for
// inequalities, [0, 0] for equalities and [-inf, ub] for the objective, is
// projected back through each operation onto its operands and finally onto
// the variables. Up to `passes` rounds, fewer when a round leaves the box
// unchanged. Returns 1 when some intersection is empty (no point of the box
// is feasible with f <= ub); otherwise 0 with the box tightened in place
// (never widened).
int host_propagate(const HostTape& H, double* box, double ub, int passes);

}  // namespace ivb
