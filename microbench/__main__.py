import json

from . import measure

print(json.dumps(measure()))
