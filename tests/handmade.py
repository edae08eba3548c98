"""Hand-built scenarios and states shared by the oracle pins and the GPU
parity tests (inputs only: no simulation arithmetic here)."""
import numpy as np

from paper_2406_10661_gb300 import scenario as sc


def one_road(n_lanes, length, cars, vmax=13.89, params=None):
    """One road of n_lanes lanes (lane 0 leftmost) and `length` metres, no
    junctions; every car drives a single-road route.  cars: list of
    (lane, s, v) or (lane, s, v, v0f).  Returns (scenario, state dict) with
    every car active at step 0; car k has vehicle id k."""
    net = sc.corridor_network(n_lanes, (length,), vmax=vmax)
    n = len(cars)
    lanes = np.array([c[0] for c in cars], dtype=np.int32)
    v0f = np.array([c[3] if len(c) > 3 else 1.0 for c in cars], dtype=np.float32)
    veh = sc.Vehicles(n=n, route_off=np.arange(n + 1, dtype=np.int32),
                      routes=np.zeros(n, dtype=np.int32), start_lane=lanes,
                      dep=np.zeros(n, dtype=np.int32), v0f=v0f)
    prm = params if params is not None else sc.Params()
    st = dict(status=np.ones(n, dtype=np.int32), lane=lanes.copy(),
              s=np.array([c[1] for c in cars], dtype=np.float64),
              v=np.array([c[2] for c in cars], dtype=np.float64),
              rc=np.zeros(n, dtype=np.int32))
    return sc.Scenario(net, veh, prm, "one_road"), st


def corridor(lengths, cars, n_lanes=1, green=30, amber=3, vmax=13.89, params=None,
             turn_len=10.0):
    """A signalised corridor; cars = list of (start_lane, dep) driving all roads."""
    net = sc.corridor_network(n_lanes, tuple(lengths), vmax=vmax, green=green, amber=amber,
                              turn_len=turn_len)
    veh = sc.corridor_vehicles(net, [c[0] for c in cars], [c[1] for c in cars])
    prm = params if params is not None else sc.Params()
    return sc.Scenario(net, veh, prm, "corridor")
