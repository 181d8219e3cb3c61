"""GB300-native spatial statistics (kNN / RDF) for atom-probe point clouds."""
from __future__ import annotations


def bins_from_spec(start: float, step: float, stop: float):
    """The paper's bin notation r = [start, step, stop] (nm) -> (r0, dr, n_bins).

    n_bins = round((stop - start) / step) in double; r0 and dr stay double so
    that edges such as 0.25 nm on a 0.01 nm step are exact.
    """
    if not (step > 0) or not (stop > start) or start < 0:
        raise ValueError("need 0 <= start < stop and step > 0")
    return float(start), float(step), int(round((stop - start) / step))
