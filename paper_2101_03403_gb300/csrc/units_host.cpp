// C ABI: functional-unit netlists (host side; no device work).
#include "ce_internal.h"
#include "netlist.h"

using namespace ce;

extern "C" ce_status ce_unit_info(int unit, int cond, int width, int *n_inputs, int *n_outputs,
                                  int *n_gates, int *n_bootstraps, int *depth) {
  Netlist n;
  if (!build_unit(unit, width, cond, &n)) return set_error(CE_EINVAL, "ce_unit_info: bad unit");
  if (n_inputs) *n_inputs = n.n_inputs;
  if (n_outputs) *n_outputs = static_cast<int>(n.outputs.size());
  if (n_gates) *n_gates = static_cast<int>(n.gates.size());
  if (n_bootstraps) *n_bootstraps = n.bootstraps();
  if (depth) *depth = n.depth;
  return CE_OK;
}

extern "C" ce_status ce_unit_netlist(int unit, int cond, int width, int32_t *buf, size_t cap,
                                     size_t *used) {
  Netlist n;
  if (!build_unit(unit, width, cond, &n)) return set_error(CE_EINVAL, "ce_unit_netlist: bad unit");
  const size_t need = 5 + 9 * n.gates.size() + 2 * n.outputs.size();
  if (used) *used = need;
  if (!buf) return CE_OK;
  if (cap < need) return set_error(CE_EINVAL, "ce_unit_netlist: buffer too small");
  size_t k = 0;
  buf[k++] = n.n_inputs;
  buf[k++] = n.n_wires;
  buf[k++] = n.depth;
  buf[k++] = static_cast<int32_t>(n.gates.size());
  buf[k++] = static_cast<int32_t>(n.outputs.size());
  for (const auto &g : n.gates) {
    buf[k++] = g.op;
    buf[k++] = g.a.wire;
    buf[k++] = g.a.neg;
    buf[k++] = g.b.wire;
    buf[k++] = g.b.neg;
    buf[k++] = g.op == kOpMux ? g.c.wire : -1;
    buf[k++] = g.op == kOpMux ? g.c.neg : 0;
    buf[k++] = g.out;
    buf[k++] = g.level;
  }
  for (const auto &r : n.outputs) {
    buf[k++] = r.wire;
    buf[k++] = r.neg;
  }
  return CE_OK;
}
