// Internal declarations of libqedpic shared by the host and device sources.
#pragma once

#include <stdint.h>

#include "qedpic.h"

namespace qp {

// Table grids (the specification published in qedpic.h).
constexpr int kNRate = QP_NRATE;        // rate nodes, 32 per octave over [2^-14, 2^10]
constexpr int kNRatePad = 776;          // device rows padded to a multiple of 16 bytes
constexpr int kRatePerOct = 32;
constexpr int kNCdf = QP_NCDF;          // CDF rows, 4 per octave over [2^-14, 2^10]
constexpr int kCdfPerOct = 4;
constexpr int kNNode = QP_NNODE;        // logit nodes per CDF row
constexpr int kChiExp0 = -14;           // first node 2^-14
constexpr int kChiExpEnd = 10;          // last node 2^10
constexpr double kSgMin = -30.0, kSgSpan = 50.0;  // emission logit nodes
constexpr double kSpMin = -20.0, kSpSpan = 40.0;  // pair logit nodes
constexpr double kPairChiMin = 0x1.0p-8;          // pair rate taken as 0 below

// Host-side FP64 tables (built by build_tables_host).
struct HostTables {
    double H[kNRate], Gs[kNRate], Ts[kNRate];
    double Cg[kNCdf * kNNode], Cp[kNCdf * kNNode];
};

// Physical constants in the context's normalised units.
struct Units {
    double a_S;     // Schwinger field / (m c omega / e)
    double C_rate;  // alpha / (sqrt(3) pi tau_c omega)
    double tau0w;   // Sokolov tau_0 * omega
};

void units_for_wavelength(double lambda_m, Units *u);
void build_tables_host(HostTables *t);

}  // namespace qp
