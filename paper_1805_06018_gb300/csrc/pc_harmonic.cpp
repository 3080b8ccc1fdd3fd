// Harmonic weights on 2D leaves that carry hanging nodes (Section 2.4).
#include "pc_internal.h"

namespace pc {

pc_status harmonic_cell_2d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err) {
    (void)g;
    (void)c;
    (void)k;
    vals.clear();
    err = "grids with hanging nodes are not supported yet";
    return PC_ERR_UNSUPPORTED;
}

}  // namespace pc
