"""Write closed_forms.json: expected colours from closed forms, using only
the math module (no oracle, no kernel).

uniform_medium_axis: a camera at (0, 0, 3) looking down -z through a single
pixel centre gives the ray along the z axis; it crosses the box [-1, 1]^3 over
a chord L = 2, i.e. G voxel sides.  With constant colour c and opacity sigma
(per voxel side) in every voxel and no shells, Eq. 3-4 telescope to
H^ = c (1 - e^{-sigma G}).
"""
import json
import math
import os

cases = []
for G, c, sigma in [(4, [0.2, 0.4, 0.6], 0.3), (8, [1.0, 0.5, 0.0], 0.05),
                    (16, [0.9, 0.1, 0.3], 1.7), (2, [0.33, 0.66, 0.99], 0.0)]:
    a = 1.0 - math.exp(-sigma * G)
    cases.append({"G": G, "c": c, "sigma": sigma,
                  "expected_rgb": [a * ci for ci in c],
                  "closed_form": "c * (1 - exp(-sigma * G))"})

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
with open(out, "w") as f:
    json.dump({"source": "PERF Eq. 3-4 (discrete volume rendering), uniform medium",
               "uniform_medium_axis": cases}, f, indent=1)
print(out)
