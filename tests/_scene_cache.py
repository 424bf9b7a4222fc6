"""Disk cache of generated test scenes (the 33.6M-triangle scene takes most of
a minute to generate).  Test helper only; the cache lives in the system temp
directory and is keyed by the generator arguments."""
import hashlib
import os
import tempfile

import numpy as np

from paper_2503_01074_gb300 import scenes as S


def cached(name, fn, *args, **kwargs):
    key = hashlib.sha256(repr((name, args, sorted(kwargs.items()))).encode()).hexdigest()[:16]
    d = os.path.join(tempfile.gettempdir(), "sonar_scene_cache")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, f"{name}_{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return S.Mesh(z["verts"], z["tris"], z["mat"]), z["mu"]
    mesh, mu, _ = fn(*args, **kwargs)
    tmp = path + f".{os.getpid()}.npz"
    np.savez(tmp, verts=mesh.verts, tris=mesh.tris, mat=mesh.mat, mu=mu)
    os.replace(tmp, path)
    return mesh, mu
