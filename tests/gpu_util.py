"""Helpers shared by the GPU tests: build/load the library, build matching
oracle and GPU media from one synthetic problem."""
import numpy as np

import oracle as O


def hz_module():
    from paper_2409_16172_gb300 import build
    build.build()
    from paper_2409_16172_gb300 import hz
    return hz


def media(hz, p, alpha=0.15, symbol_kind=0, a_node=0.0, M=None, Mt=None, oracle=True, Ma=0,
          basis=0):
    M = p.M if M is None else M
    Mt = p.Mt if Mt is None else Mt
    med_g = hz.Medium(p.c, p.zeta if np.any(p.zeta > 0) else None, p.a, omega=p.omega, M=M, Mt=Mt,
                      c_o=p.c_o, alpha=alpha, a_node=a_node, symbol_kind=symbol_kind, Ma=Ma,
                      basis=basis)
    med_o = None
    if oracle:
        med_o = O.make_medium(p.c, p.zeta, p.a, p.omega, M, Mt, p.c_o, None, alpha, a_node,
                              symbol_kind, Ma=max(Ma, 1), basis=basis)
    return med_g, med_o


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
