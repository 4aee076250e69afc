// Host-side construction of a system's force-field parameters, shared by
// mdas_create_system and mdas_forces_noalloc so that both evaluate the same
// force field from the same description.  Not part of the public ABI.
#pragma once
#include "../../include/mdas.h"
#include "mdas_dev.cuh"

namespace mdas {

// The force-field part of P from a description (Sec. 3): sizes, the box and
// its derived fields, a cell grid of edge >= rc for every box edge shrunk to
// (1 - shrink) of its length, the cutoff and reaction-field constants, the
// pair tables, the bead types of every lipid type and the bonded topology
// (bonds, angles, exclusions, bonded partners).  P is cleared first; the
// caller adds capacities, the pair list and the thermostat.  Returns nullptr
// on success, else a one-line reason (the description is invalid).
const char *fill_force_field(const mdas_system_desc *d, double shrink, Params &P);

}  // namespace mdas
