// Gate matrices of the Sycamore-class gate set, in FP64, and gate validation.
//
// The paper uses Google's Sycamore circuits (Section 3.1) without writing their
// gates down. The matrices here are the principal square roots of X, Y and
// W = (X + Y)/sqrt(2), and fSim(theta, phi), written out entry by entry:
//   sqrtX = 1/2 [[1+i, 1-i], [1-i, 1+i]]
//   sqrtY = 1/2 [[1+i, -1-i], [1+i, 1+i]]
//   sqrtW = [[(1+i)/2, -i/sqrt2], [1/sqrt2, (1+i)/2]]
//   fSim  = [[1,0,0,0],[0,cos t,-i sin t,0],[0,-i sin t,cos t,0],[0,0,0,e^{-i phi}]]
#include <cmath>
#include <cstring>

#include "internal.h"

namespace rcs {

static void adjoint_inplace(cd *m, int d) {
    cd t[16];
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) t[r * d + c] = std::conj(m[c * d + r]);
    std::memcpy(static_cast<void *>(m), t, sizeof(cd) * d * d);
}

static double unitarity_defect(const cd *m, int d) {
    double worst = 0.0;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            cd s = 0.0;
            for (int l = 0; l < d; ++l) s += m[r * d + l] * std::conj(m[c * d + l]);
            worst = std::fmax(worst, std::abs(s - (r == c ? 1.0 : 0.0)));
        }
    return worst;
}

int gate_to_host(const rcs_gate &g, int n, HostGate *out, std::string *why) {
    const cd i1(0.0, 1.0);
    const double h = 0.5, rs2 = 1.0 / std::sqrt(2.0);
    int nq;
    switch (g.kind) {
        case RCS_GATE_SQRT_X:
            nq = 1;
            out->m[0] = h * cd(1, 1);
            out->m[1] = h * cd(1, -1);
            out->m[2] = h * cd(1, -1);
            out->m[3] = h * cd(1, 1);
            break;
        case RCS_GATE_SQRT_Y:
            nq = 1;
            out->m[0] = h * cd(1, 1);
            out->m[1] = h * cd(-1, -1);
            out->m[2] = h * cd(1, 1);
            out->m[3] = h * cd(1, 1);
            break;
        case RCS_GATE_SQRT_W:
            nq = 1;
            out->m[0] = h * cd(1, 1);
            out->m[1] = cd(0, -rs2);
            out->m[2] = cd(rs2, 0);
            out->m[3] = h * cd(1, 1);
            break;
        case RCS_GATE_FSIM: {
            nq = 2;
            for (int e = 0; e < 16; ++e) out->m[e] = 0.0;
            const double c = std::cos(g.theta), s = std::sin(g.theta);
            out->m[0] = 1.0;
            out->m[5] = c;
            out->m[6] = -i1 * s;
            out->m[9] = -i1 * s;
            out->m[10] = c;
            out->m[15] = std::exp(-i1 * g.phi);
            break;
        }
        case RCS_GATE_U1:
        case RCS_GATE_U2: {
            nq = g.kind == RCS_GATE_U1 ? 1 : 2;
            if (!g.u) {
                *why = "U1/U2 gate without a matrix";
                return RCS_ERR_ARG;
            }
            const int d = 1 << nq;
            for (int e = 0; e < d * d; ++e) out->m[e] = cd(g.u[2 * e], g.u[2 * e + 1]);
            if (!(unitarity_defect(out->m, d) <= 1e-6)) {
                *why = "U1/U2 matrix is not unitary to 1e-6";
                return RCS_ERR_ARG;
            }
            break;
        }
        default:
            *why = "unknown gate kind " + std::to_string(int(g.kind));
            return RCS_ERR_ARG;
    }
    if (g.nq != nq) {
        *why = "gate nq does not match its kind";
        return RCS_ERR_ARG;
    }
    for (int i = 0; i < nq; ++i) {
        if (g.q[i] < 0 || g.q[i] >= n) {
            *why = "qubit " + std::to_string(g.q[i]) + " out of range for " + std::to_string(n) + " qubits";
            return RCS_ERR_QUBIT;
        }
        out->q[i] = g.q[i];
    }
    if (nq == 2 && g.q[0] == g.q[1]) {
        *why = "two-qubit gate with repeated qubit";
        return RCS_ERR_QUBIT;
    }
    if (nq == 1) out->q[1] = -1;
    out->nq = nq;
    if (g.flags & RCS_FLAG_ADJOINT) adjoint_inplace(out->m, 1 << nq);
    return RCS_OK;
}

}  // namespace rcs
