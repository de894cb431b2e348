"""The vehicle loop's backend over the CPU oracle (test infrastructure): the same colony, road model and
tick as the library, so a simulation on it must match one on the library step for step."""
import numpy as np


class OracleBackend:
    def __init__(self, orc, wl, flags=0):
        self.orc = orc
        self.net = wl.net
        self.sig = wl.signals
        self.flags = flags
        self.veh = np.zeros(wl.net.n_edges, np.uint32)
        self.red = np.zeros((wl.net.n_nodes, 8), np.uint32)
        self.order = orc.queue_preempt(self._onet())

    def _onet(self):
        return self.orc.Net(self.net, self.sig, self.veh, self.red)

    def set_densities(self, veh):
        self.veh = np.array(veh, np.uint32)
        self.order = self.orc.queue_preempt(self._onet())

    def road_state(self):
        prep = self.orc.prepare(self._onet(), self.orc.Params(), 0)
        return prep["tt"], prep["qd"], self.order

    def route_batch(self, t_ms, queries):
        onet = self._onet()
        prm = self.orc.Params(t_dep_ms=t_ms, flags=self.flags)
        out = []
        for q in queries:
            r = self.orc.solve(onet, prm, q, want_tau=False)
            out.append((r["status"], r["route"]))
        return out

    def tick(self, t_ms, dt_ms):
        self.veh, self.red, self.order = self.orc.tick(self._onet(), self.orc.Params(), t_ms, dt_ms, self.order)
