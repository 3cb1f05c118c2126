// The device-resident state of one conjugate-gradient segment, shared by the
// CG kernels (solve.cu) and the multigrid preconditioner (mg.cu).
#pragma once

#include "internal.cuh"

namespace osm {

enum { kRunning = 0, kConverged = 1, kFinished = 2 };

struct CgState {
    double rho, rho0, pq, alpha, beta, stop2;
    double rr;         // preconditioned CG: |r|^2, the stopping test (rho is then (r, z))
    long long it, max_it;
    int status, first, breakdown, err;  // err: a bounded device-side wait ran out
    int precond;       // 1: z = B r by the multigrid preconditioner before every direction update
    int pending;       // preconditioned CG: the segment's first (r, z) is still to be formed
    int keep;          // ... and the previous search direction is kept (reliable-update continuation)
    int loops;         // bodies run by the device-side CG loop in this graph launch
    unsigned ticketA, ticketB, ticketI, ticketM;
};

}  // namespace osm
